"""Legendre functions for the oracle (test infrastructure only).

Off the cut (Sec. 2.3, "Legendre function evaluation"):
  * x > 1 real (prolate) or x = i*u, u > 0 (oblate).
  * Convention: Hobson's type 3,  P_n^m(x) = (x^2-1)^{m/2} d^m P_n/dx^m  and
    Q_n^m(x) = (x^2-1)^{m/2} d^m Q_n/dx^m, with Q_0(x) = 1/2 log((x+1)/(x-1)).
    For complex x the root (x^2-1)^{1/2} is the product of the principal roots
    (x+1)^{1/2} (x-1)^{1/2}, so that (x^2-1)^{1/2} = i sqrt(u^2+1) at x = i u.
    With this convention P_m^m = (2m-1)!! (x^2-1)^{m/2} exactly as printed in
    Sec. 2.3, and the Casoratian of eq. (PQ) holds with the printed sign.
  * P by the forward three-term recurrence, eq. (recur), step 1.
  * Q by the paper's steps 2-4: for every order m the ratio
    H_N^m = Q_N^m / Q_{N-1}^m from the continued fraction eq.
    (continuedfraction) evaluated with the modified Lentz method; Q_{N-1}^m
    and Q_N^m from eqs. (QfromP1), (QfromP2) (the Casoratian, eq. (PQ), at
    n = N); then the recurrence run backwards to n = m.
  * First derivatives from eq. (derivative), which both families satisfy.

On the cut (Definition 1): Ferrers functions Pbar_n^m(v) = (1-v^2)^{m/2}
d^m P_n/dv^m (no Condon-Shortley phase) and the real orthonormal surface
harmonics built from them.

Readings of the paper taken here (the paper is silent on them):
  * Lentz tolerance |Delta - 1| < 4e-16 (two ulps of 1), at most 10^4 terms,
    tiny = 1e-300.
  * The printed constant of eq. (QfromP1) has a lower-case n; it is read as
    the truncation index N (the Casoratian is used at n = N).
"""
from __future__ import annotations

import math

import numpy as np

LENTZ_TOL = 4e-16
LENTZ_MAXIT = 10000
LENTZ_TINY = 1e-300


def _sqrt_xm1xp1(x):
    """(x^2-1)^{1/2} as (x+1)^{1/2} (x-1)^{1/2} with principal roots."""
    if np.iscomplexobj(x):
        return np.sqrt(x + 1.0) * np.sqrt(x - 1.0)
    return np.sqrt(x + 1.0) * np.sqrt(x - 1.0)


def double_factorial_odd(m: int) -> float:
    """(2m-1)!! with (-1)!! = 1."""
    r = 1.0
    for k in range(1, 2 * m, 2):
        r *= k
    return r


def legendre_P(x, N: int):
    """P_n^m(x) for 0 <= m <= n <= N, array of shape x.shape + (N+1, N+1)
    indexed [..., n, m] (zero where m > n).  Sec. 2.3 step 1."""
    x = np.asarray(x)
    dt = np.complex128 if np.iscomplexobj(x) else np.float64
    x = x.astype(dt)
    P = np.zeros(x.shape + (N + 1, N + 1), dtype=dt)
    s = _sqrt_xm1xp1(x)
    for m in range(N + 1):
        Pmm = double_factorial_odd(m) * s ** m
        P[..., m, m] = Pmm
        if m + 1 <= N:
            P[..., m + 1, m] = x * (2 * m + 1) * Pmm
        for n in range(m + 1, N):
            # eq. (recur): (n-m+1) P_{n+1} = (2n+1) x P_n - (n+m) P_{n-1}
            P[..., n + 1, m] = ((2 * n + 1) * x * P[..., n, m] - (n + m) * P[..., n - 1, m]) / (n - m + 1)
    return P


def continued_fraction_H(x, n0: int, m: int):
    """H_{n0}^m(x) = Q_{n0}^m / Q_{n0-1}^m from eq. (continuedfraction),
    H_n = a_n / (b_n + H_{n+1}), a_n = -(n+m)/(n-m+1), b_n = -(2n+1)x/(n-m+1),
    evaluated with the modified Lentz method (f = b_0 + a_1/(b_1 + ...),
    here with b_0 = 0).  Returns (H, iterations used)."""
    x = np.asarray(x)
    dt = np.complex128 if np.iscomplexobj(x) else np.float64
    x = x.astype(dt)
    f = np.full(x.shape, LENTZ_TINY, dtype=dt)
    C = f.copy()
    D = np.zeros(x.shape, dtype=dt)
    done = np.zeros(x.shape, dtype=bool)
    for it in range(1, LENTZ_MAXIT + 1):
        n = n0 + it - 1
        a = -(n + m) / (n - m + 1.0)
        b = -(2 * n + 1) * x / (n - m + 1.0)
        D = b + a * D
        D = np.where(D == 0, LENTZ_TINY, D)
        C = b + a / C
        C = np.where(C == 0, LENTZ_TINY, C)
        D = 1.0 / D
        delta = C * D
        f = np.where(done, f, f * delta)
        done |= np.abs(delta - 1.0) < LENTZ_TOL
        if np.all(done):
            return f, it
    raise RuntimeError("continued fraction for H_N^m did not converge")


def legendre_Q(x, N: int, P=None):
    """Q_n^m(x) for 0 <= m <= n <= N, shape x.shape + (N+1, N+1), by the
    steps 2-4 of Sec. 2.3 (needs N >= 1)."""
    if N < 1:
        raise ValueError("legendre_Q needs N >= 1")
    x = np.asarray(x)
    dt = np.complex128 if np.iscomplexobj(x) else np.float64
    x = x.astype(dt)
    if P is None:
        P = legendre_P(x, N)
    Q = np.zeros(x.shape + (N + 1, N + 1), dtype=dt)
    for m in range(N + 1):
        H, _ = continued_fraction_H(x, N, m)
        casor = math.factorial(N + m - 1) / math.factorial(N - m) * (-1.0) ** m
        PNm1 = P[..., N - 1, m] if N - 1 >= m else np.zeros(x.shape, dtype=dt)
        QNm1 = casor / (P[..., N, m] - H * PNm1)          # eq. (QfromP1)
        QN = H * QNm1                                      # eq. (QfromP2)
        Q[..., N, m] = QN
        if N - 1 >= m:
            Q[..., N - 1, m] = QNm1
        # backward recurrence: Q_{n-1} = ((2n+1) x Q_n - (n-m+1) Q_{n+1}) / (n+m)
        for n in range(N - 1, m, -1):
            Q[..., n - 1, m] = ((2 * n + 1) * x * Q[..., n, m] - (n - m + 1) * Q[..., n + 1, m]) / (n + m)
    return Q


def derivative(F, x, N: int):
    """First derivatives d/dx of F_n^m (F = P or Q arrays reaching n = N+1),
    from eq. (derivative): (1-x^2) F_n' = (m-n-1) F_{n+1} + (n+1) x F_n.
    Returns shape x.shape + (N+1, N+1)."""
    x = np.asarray(x)
    dF = np.zeros(F.shape[:-2] + (N + 1, N + 1), dtype=F.dtype)
    for n in range(N + 1):
        for m in range(n + 1):
            dF[..., n, m] = ((m - n - 1) * F[..., n + 1, m] + (n + 1) * x * F[..., n, m]) / (1.0 - x * x)
    return dF


def legendre_PQ_with_derivatives(x, N: int):
    """P, Q, P', Q' for n, m <= N (computing one order further for eq. (derivative))."""
    x = np.asarray(x)
    P = legendre_P(x, N + 1)
    Q = legendre_Q(x, N + 1, P)
    dP = derivative(P, x, N)
    dQ = derivative(Q, x, N)
    return P[..., :N + 1, :N + 1], Q[..., :N + 1, :N + 1], dP, dQ


# ----------------------------------------------------------------------------
# on the cut: Ferrers functions and the real surface-harmonic basis
# ----------------------------------------------------------------------------

def norm_factor(n: int, m: int) -> float:
    """N_n^m = sqrt((2n+1)/(4 pi) (n-m)!/(n+m)!), Definition 1."""
    return math.sqrt((2 * n + 1) / (4 * math.pi) * math.factorial(n - m) / math.factorial(n + m))


def ferrers_P(v, N: int):
    """Ferrers Pbar_n^m(v), |v| <= 1, no Condon-Shortley phase; [..., n, m]."""
    v = np.asarray(v, dtype=np.float64)
    P = np.zeros(v.shape + (N + 1, N + 1))
    s = np.sqrt(np.maximum(1.0 - v * v, 0.0))
    for m in range(N + 1):
        P[..., m, m] = double_factorial_odd(m) * s ** m
        if m + 1 <= N:
            P[..., m + 1, m] = v * (2 * m + 1) * P[..., m, m]
        for n in range(m + 1, N):
            P[..., n + 1, m] = ((2 * n + 1) * v * P[..., n, m] - (n + m) * P[..., n - 1, m]) / (n - m + 1)
    return P


def coeff_index(n: int, m: int) -> int:
    return n * n + n + m


def real_Y(v, phi, p: int):
    """Real orthonormal surface harmonics at (v, phi), shape v.shape + ((p+1)^2,):
       m > 0: sqrt(2) N_n^m Pbar_n^m(v) cos(m phi)
       m = 0: N_n^0 P_n(v)
       m < 0: sqrt(2) N_n^|m| Pbar_n^|m|(v) sin(|m| phi)
    orthonormal for  int_{-1}^{1} int_0^{2 pi} . dphi dv  (Definition 1)."""
    v = np.asarray(v, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    P = ferrers_P(v, p)
    Y = np.zeros(np.broadcast(v, phi).shape + ((p + 1) ** 2,))
    for n in range(p + 1):
        for m in range(-n, n + 1):
            am = abs(m)
            base = norm_factor(n, am) * P[..., n, am]
            if m > 0:
                Y[..., coeff_index(n, m)] = math.sqrt(2.0) * base * np.cos(am * phi)
            elif m < 0:
                Y[..., coeff_index(n, m)] = math.sqrt(2.0) * base * np.sin(am * phi)
            else:
                Y[..., coeff_index(n, m)] = base
    return Y


def abs_m_table(p: int):
    """(n, |m|) of every coefficient index, for broadcasting multipliers."""
    ns, ms = [], []
    for n in range(p + 1):
        for m in range(-n, n + 1):
            ns.append(n)
            ms.append(abs(m))
    return np.array(ns), np.array(ms)
