"""Seeded synthetic workloads for the spheroidal boundary-integral apply.

This module only *draws inputs*: spheroid shapes, placements, orientations and
spheroidal-harmonic coefficient vectors.  It contains none of the method's
arithmetic (no Legendre functions, no layer-potential multipliers, no
quadrature, no near/far classification), so both the CPU oracle and the CUDA
path can consume its output without sharing any computation.

Spheroid descriptor (one row per particle), following the problem statement of
Sec. 5.1 (shape type, semi-axes, centre, unit quaternion):

    kind   0 = prolate (C > A), 1 = oblate (C < A)
    A      equatorial semi-axis (radius of the circular cross-section), Sec. 2.1
    C      polar semi-axis (along the local x3 axis), Sec. 2.1
    center (3,) global position of the centre
    quat   (4,) unit quaternion (w, x, y, z); x_global = center + R(quat) x_local

Coefficient vectors use the real orthonormal surface-harmonic basis indexed by
``n*n + n + m`` for 0 <= n <= p, -n <= m <= n (m > 0 cosine, m < 0 sine).

The placement code below needs a spheroid-spheroid separation test.  It uses
its own sampled point-to-ellipse distance (bisection on the Lagrange
parameter); it decides only whether a drawn configuration is admissible and is
never used to compute an operator value.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

PROLATE = 0
OBLATE = 1


@dataclasses.dataclass
class Suspension:
    """A set of M spheroids plus the discretisation order used with it."""

    kind: np.ndarray      # (M,) int32
    A: np.ndarray         # (M,) float64
    C: np.ndarray         # (M,) float64
    center: np.ndarray    # (M, 3) float64
    quat: np.ndarray      # (M, 4) float64, unit, (w, x, y, z)
    p: int
    name: str = ""

    @property
    def M(self) -> int:
        return int(self.kind.shape[0])

    def subset(self, idx) -> "Suspension":
        idx = np.asarray(idx)
        return Suspension(self.kind[idx].copy(), self.A[idx].copy(), self.C[idx].copy(),
                          self.center[idx].copy(), self.quat[idx].copy(), self.p, self.name)


# ----------------------------------------------------------------------------
# random primitives
# ----------------------------------------------------------------------------

def random_quaternions(rng: np.random.Generator, M: int) -> np.ndarray:
    """Uniform random rotations: normalised 4-D Gaussian vectors."""
    q = rng.standard_normal((M, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def coefficients(rng: np.random.Generator, M: int, p: int, ndens: int = 1) -> np.ndarray:
    """i.i.d. N(0,1)/(n+1)^2 coefficients, shape (M, ndens, (p+1)^2) squeezed
    to (M, (p+1)^2) when ndens == 1."""
    nc = (p + 1) ** 2
    n_of = np.floor(np.sqrt(np.arange(nc))).astype(np.int64)
    scale = 1.0 / (n_of + 1.0) ** 2
    c = rng.standard_normal((M, ndens, nc)) * scale
    return c[:, 0, :] if ndens == 1 else c


def _quat_to_matrix(q: np.ndarray) -> np.ndarray:
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.empty(q.shape[:-1] + (3, 3))
    R[..., 0, 0] = 1 - 2 * (y * y + z * z)
    R[..., 0, 1] = 2 * (x * y - w * z)
    R[..., 0, 2] = 2 * (x * z + w * y)
    R[..., 1, 0] = 2 * (x * y + w * z)
    R[..., 1, 1] = 1 - 2 * (x * x + z * z)
    R[..., 1, 2] = 2 * (y * z - w * x)
    R[..., 2, 0] = 2 * (x * z - w * y)
    R[..., 2, 1] = 2 * (y * z + w * x)
    R[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return R


# ----------------------------------------------------------------------------
# separation test used only to accept / reject a drawn placement
# ----------------------------------------------------------------------------

def _ellipse_gap(r, z, A, C):
    """Signed distance from meridian-plane points (r >= 0, z >= 0) to the
    ellipse r^2/A^2 + z^2/C^2 = 1; negative inside.  For exterior points the
    closest point is x = (A^2 r/(t+A^2), C^2 z/(t+C^2)) with t >= 0 the root of
    the convex decreasing F(t) = (A r/(t+A^2))^2 + (C z/(t+C^2))^2 - 1;
    Newton's method from t = 0 approaches it monotonically from the left."""
    r = np.asarray(r, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    inside = (r / A) ** 2 + (z / C) ** 2 < 1.0
    ar, cz = A * r, C * z
    A2, C2 = A * A, C * C
    t = np.zeros_like(r)
    for _ in range(40):
        ea, ec = ar / (t + A2), cz / (t + C2)
        F = ea * ea + ec * ec - 1.0
        dF = -2.0 * (ea * ea / (t + A2) + ec * ec / (t + C2))
        step = np.where(inside | (dF == 0.0), 0.0, F / np.where(dF == 0.0, 1.0, dF))
        t = t - step
        if np.all(np.abs(step) <= 1e-15 * (np.abs(t) + 1e-300)):
            break
    xr = A2 * r / (t + A2)
    xz = C2 * z / (t + C2)
    d = np.hypot(r - xr, z - xz)
    return np.where(inside, -1.0, d)


def _surface_points(A, C, theta, phi):
    st = np.sin(theta)
    return np.stack([A * st * np.cos(phi), A * st * np.sin(phi), C * np.cos(theta)], axis=-1)


def _gap_one_way(Ai, Ci, ci, Ri, Aj, Cj, cj, Rj):
    """min over sampled points of spheroid i of the signed distance to spheroid j,
    with three rounds of local refinement around the best sample."""
    def dist_of(theta, phi):
        x = _surface_points(Ai, Ci, theta, phi) @ Ri.T + ci      # global
        xl = (x - cj) @ Rj                                         # j-local
        rr = np.hypot(xl[..., 0], xl[..., 1])
        return _ellipse_gap(rr, np.abs(xl[..., 2]), Aj, Cj)

    th = np.linspace(0.0, np.pi, 13)
    ph = np.linspace(0.0, 2 * np.pi, 24, endpoint=False)
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    d = dist_of(TH, PH)
    k = np.unravel_index(np.argmin(d), d.shape)
    best, bt, bp = d[k], TH[k], PH[k]
    h_t, h_p = np.pi / 12, 2 * np.pi / 24
    for _ in range(6):
        lt = bt + h_t * np.linspace(-1, 1, 7)
        lp = bp + h_p * np.linspace(-1, 1, 7)
        TT, PP = np.meshgrid(np.clip(lt, 0, np.pi), lp, indexing="ij")
        dd = dist_of(TT, PP)
        kk = np.unravel_index(np.argmin(dd), dd.shape)
        if dd[kk] < best:
            best, bt, bp = dd[kk], TT[kk], PP[kk]
        h_t /= 3.0
        h_p /= 3.0
    return float(np.min(d)) if np.min(d) < 0 else float(best)


def separation(s: Suspension, i: int, j: int, R=None) -> float:
    """Estimated surface gap between spheroids i and j (<= 0 means overlap)."""
    if R is None:
        R = _quat_to_matrix(s.quat)
    g1 = _gap_one_way(s.A[i], s.C[i], s.center[i], R[i], s.A[j], s.C[j], s.center[j], R[j])
    if g1 < 0:
        return g1
    g2 = _gap_one_way(s.A[j], s.C[j], s.center[j], R[j], s.A[i], s.C[i], s.center[i], R[i])
    return min(g1, g2)


def _admissible(kind, A, C, center, R, new, placed, min_gap):
    """True if spheroid `new` keeps a gap >= min_gap to every index in `placed`."""
    if len(placed) == 0:
        return True
    placed = np.asarray(placed)
    d = np.linalg.norm(center[placed] - center[new], axis=1)
    rmax = np.maximum(A, C)
    rmin = np.minimum(A, C)
    if np.any(d - rmin[placed] - rmin[new] < min_gap):
        return False
    amb = placed[d - rmax[placed] - rmax[new] < min_gap]
    if len(amb):
        # separating-axis bound along the centre line: the gap is at least the
        # centre distance minus both support functions in that direction
        u = (center[new] - center[amb]) / np.linalg.norm(center[new] - center[amb], axis=1, keepdims=True)
        ax_new = R[new][:, 2]
        ax_amb = R[amb][:, :, 2]

        def support(Aa, Cc, cos_t):
            return np.sqrt(Aa * Aa + (Cc * Cc - Aa * Aa) * cos_t * cos_t)

        lb = (np.linalg.norm(center[new] - center[amb], axis=1) - support(A[new], C[new], u @ ax_new)
              - support(A[amb], C[amb], np.sum(u * ax_amb, axis=1)))
        amb = amb[lb < min_gap]
    for j in amb:
        g1 = _gap_one_way(A[new], C[new], center[new], R[new], A[j], C[j], center[j], R[j])
        if g1 < min_gap:
            return False
        g2 = _gap_one_way(A[j], C[j], center[j], R[j], A[new], C[new], center[new], R[new])
        if g2 < min_gap:
            return False
    return True


# ----------------------------------------------------------------------------
# workload recipes
# ----------------------------------------------------------------------------

def lattice_suspension(seed: int = 0, p: int = 8, spacing: float = 5.0,
                       jitter: float = 0.5, min_gap: float = 0.2) -> Suspension:
    """Eight spheroids on a jittered 2x2x2 lattice: prolates (A=1, C=2) and
    oblates (A=1.5, C=0.75) alternating by lattice parity, random orientations.
    The lattice shape follows the 2x2 prolate lattice test of Sec. 5.2."""
    rng = np.random.default_rng(seed)
    idx = np.array([(i, j, k) for i in range(2) for j in range(2) for k in range(2)], dtype=np.float64)
    kind = (idx.sum(axis=1).astype(np.int64) % 2).astype(np.int32)   # 0 prolate, 1 oblate
    A = np.where(kind == PROLATE, 1.0, 1.5)
    C = np.where(kind == PROLATE, 2.0, 0.75)
    for _ in range(1000):
        center = idx * spacing + rng.uniform(-jitter, jitter, size=(8, 3))
        quat = random_quaternions(rng, 8)
        R = _quat_to_matrix(quat)
        ok = all(_admissible(kind, A, C, center, R, n, list(range(n)), min_gap) for n in range(1, 8))
        if ok:
            return Suspension(kind, A, C, center, quat, p, "lattice8")
    raise RuntimeError("could not place lattice suspension")


def random_shapes(rng: np.random.Generator, M: int, ar_range=(1.2, 5.0), major_range=(0.5, 1.5)):
    """Polydisperse spheroid shapes: aspect ratio U[ar], major semi-axis
    U[major], prolate or oblate with probability 1/2."""
    ar = rng.uniform(*ar_range, size=M)
    major = rng.uniform(*major_range, size=M)
    kind = (rng.uniform(size=M) < 0.5).astype(np.int32)     # 1 = oblate
    A = np.where(kind == PROLATE, major / ar, major)
    C = np.where(kind == PROLATE, major, major / ar)
    return kind, A, C


def rsa_suspension(M: int, phi_vol: float, seed: int, p: int, ar_range=(1.2, 5.0),
                   major_range=(0.5, 1.5), min_gap: float = 0.05, name: str = "rsa",
                   max_attempts: int = 200000) -> Suspension:
    """Random sequential addition in a cube of side L = (sum V / phi_vol)^(1/3):
    centres U[0, L]^3, uniform random orientation, rejected while the gap to
    any placed particle is below `min_gap`."""
    rng = np.random.default_rng(seed)
    kind, A, C = random_shapes(rng, M, ar_range, major_range)
    vol = 4.0 / 3.0 * np.pi * A * A * C
    L = (vol.sum() / phi_vol) ** (1.0 / 3.0)
    center = np.zeros((M, 3))
    quat = np.zeros((M, 4))
    R = np.zeros((M, 3, 3))
    attempts = 0
    for n in range(M):
        while True:
            attempts += 1
            if attempts > max_attempts:
                raise RuntimeError(f"RSA failed to place {M} particles at phi={phi_vol}")
            center[n] = rng.uniform(0.0, L, size=3)
            quat[n] = random_quaternions(rng, 1)[0]
            R[n] = _quat_to_matrix(quat[n])
            if _admissible(kind, A, C, center, R, n, list(range(n)), min_gap):
                break
    return Suspension(kind, A, C, center, quat, p, name)


def config_suspension(cfg: int, seed: int = 0) -> Suspension:
    """Suspensions of the three single-geometry workloads:
      1: 8-spheroid jittered lattice, p = 8
      2: 200 polydisperse spheroids, AR U[1.2,5], major U[0.5,1.5], 20 %, gap 0.05, p = 16
      3: 100 spheroids, AR U[1.5,4], major U[0.5,1.5], 15 %, gap 0.05, p = 12 (Stokes)
    """
    if cfg == 1:
        return lattice_suspension(seed, p=8)
    if cfg == 2:
        return rsa_suspension(200, 0.20, seed, p=16, ar_range=(1.2, 5.0), name="poly200")
    if cfg == 3:
        return rsa_suspension(100, 0.15, seed, p=12, ar_range=(1.5, 4.0), name="stokes100")
    raise ValueError(cfg)


def config_coefficients(s: Suspension, seed: int = 0, ndens: int = 2) -> np.ndarray:
    """Coefficient sets for a suspension: (ndens, M, (p+1)^2); for the Laplace
    workloads density 0 is the single-layer input (modified basis) and density
    1 the double-layer input; for Stokes the three Cartesian components."""
    rng = np.random.default_rng([seed, 7919])
    c = coefficients(rng, s.M, s.p, ndens)
    if ndens == 1:
        return c[None]
    return np.ascontiguousarray(np.transpose(c, (1, 0, 2)))


def _batch_member(args):
    s, base_seed, p_choices, M_range, phi_range = args
    rng = np.random.default_rng([base_seed + s, 104729])
    M = int(round(math.exp(rng.uniform(math.log(M_range[0]), math.log(M_range[1])))))
    p = int(rng.choice(p_choices))
    phi = float(rng.uniform(*phi_range))
    return rsa_suspension(M, phi, base_seed + s, p, name=f"batch{s}")


def batch_suspensions(n: int = 64, base_seed: int = 0, p_choices=(8, 12, 16, 20),
                      M_range=(10, 400), phi_range=(0.05, 0.25), workers: int = 1):
    """Independent suspensions for the batched workload: suspension s uses
    seed base_seed + s; M log-uniform in M_range, p uniform over p_choices,
    volume fraction U[phi_range], shapes as the 200-particle workload.
    workers > 1 draws them in spawned processes (same result)."""
    jobs = [(s, base_seed, tuple(p_choices), tuple(M_range), tuple(phi_range)) for s in range(n)]
    if workers <= 1:
        return [_batch_member(j) for j in jobs]
    import concurrent.futures as cf
    import multiprocessing as mp

    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_batch_member, jobs))


def poisson_requests(rate: float, duration: float, seed: int = 0, M_range=(20, 500),
                     p_choices=(8, 12, 16), max_requests=None):
    """Arrival stream for the served workload: Poisson arrivals at `rate`/s for
    `duration` s; each request has M log-uniform in M_range, p from p_choices
    and is a Laplace S+D or a Stokes single-layer request with probability 1/2."""
    rng = np.random.default_rng([seed, 15485863])
    t = 0.0
    reqs = []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration or (max_requests is not None and len(reqs) >= max_requests):
            break
        M = int(round(math.exp(rng.uniform(math.log(M_range[0]), math.log(M_range[1])))))
        p = int(rng.choice(p_choices))
        op = "laplace" if rng.uniform() < 0.5 else "stokes"
        reqs.append({"t": t, "M": M, "p": p, "op": op, "seed": int(rng.integers(1 << 30))})
    return reqs


def shell_points(s: Suspension, distances=(1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6), per_particle: int = 4,
                 seed: int = 0, far_points: int = 0) -> np.ndarray:
    """Evaluation points shaped like the shell tests of the paper's numerical
    section: for every particle and every distance d, `per_particle` points
    offset by d along the outward normal of random surface points (distance
    to that surface d, or less on strongly curved parts); plus `far_points`
    points uniform in the suspension's bounding box.  Points that fall
    inside (or within 1e-9 of) any spheroid are dropped.  Returns (T, 3)."""
    rng = np.random.default_rng([seed, 271828])
    R = _quat_to_matrix(s.quat)
    pts = []
    for i in range(s.M):
        for d in distances:
            th = np.arccos(rng.uniform(-1.0, 1.0, per_particle))
            ph = rng.uniform(0.0, 2 * math.pi, per_particle)
            xl = np.stack([s.A[i] * np.sin(th) * np.cos(ph), s.A[i] * np.sin(th) * np.sin(ph),
                           s.C[i] * np.cos(th)], -1)
            g = xl / np.array([s.A[i] ** 2, s.A[i] ** 2, s.C[i] ** 2])
            nl = g / np.linalg.norm(g, axis=1, keepdims=True)
            pts.append((xl + d * nl) @ R[i].T + s.center[i])
    if far_points:
        lo = s.center.min(0) - np.maximum(s.A, s.C).max()
        hi = s.center.max(0) + np.maximum(s.A, s.C).max()
        pts.append(rng.uniform(lo, hi, (far_points, 3)))
    X = np.concatenate(pts) if pts else np.zeros((0, 3))
    keep = np.ones(len(X), bool)
    for i in range(s.M):
        xl = (X - s.center[i]) @ R[i]
        f = (xl[:, 0] ** 2 + xl[:, 1] ** 2) / s.A[i] ** 2 + xl[:, 2] ** 2 / s.C[i] ** 2
        keep &= f > 1.0 + 1e-9
    return np.ascontiguousarray(X[keep])


def interior_charges(s: Suspension, per_particle: int = 2, seed: int = 0, spread: float = 0.05):
    """Point charges inside the particles, as in the paper's boundary-value
    tests: `per_particle` charges per spheroid at centre + R (U(-spread,
    spread)^3 * (A, A, C)), strengths U(-0.5, 0.5).  Returns (xs (K, 3), qs (K,))."""
    rng = np.random.default_rng([seed, 314159])
    R = _quat_to_matrix(s.quat)
    xs = np.concatenate([s.center[i] + (rng.uniform(-spread, spread, (per_particle, 3))
                                        * np.array([s.A[i], s.A[i], s.C[i]])) @ R[i].T for i in range(s.M)])
    return xs, rng.uniform(-0.5, 0.5, len(xs))


def elongated_pair(ar: float, kind0: int, p: int, gap: float = 0.1, tilt: float = 0.7) -> Suspension:
    """Two spheroids for the aspect-ratio tests (the paper's stress tests run
    prolates up to aspect ratio 64): particle 0 has major semi-axis 1 and
    aspect ratio `ar` (prolate: C = 1, A = 1/ar; oblate: A = 1, C = 1/ar),
    centred at the origin with the identity orientation; particle 1, a
    prolate A = 0.25, C = 0.5 tilted by `tilt` about x, sits beyond the tip
    (prolate) or the rim (oblate) of particle 0 with its centre `gap` + 0.25
    beyond it."""
    if kind0 == PROLATE:
        A0, C0 = 1.0 / ar, 1.0
        c1 = np.array([0.0, 0.0, C0 + gap + 0.25])
    else:
        A0, C0 = 1.0, 1.0 / ar
        c1 = np.array([A0 + gap + 0.25, 0.0, 0.0])
    kind = np.array([kind0, PROLATE], np.int32)
    A = np.array([A0, 0.25])
    C = np.array([C0, 0.5])
    quat = np.array([[1.0, 0.0, 0.0, 0.0], [math.cos(tilt / 2), math.sin(tilt / 2), 0.0, 0.0]])
    center = np.stack([np.zeros(3), c1])
    return Suspension(kind, A, C, center, quat, p, f"elongated{ar:g}")


def extreme_points(s: Suspension, i: int, distances=(1e-1, 1e-2, 1e-3), n_side: int = 8) -> np.ndarray:
    """Points at distance d outside the most curved and the flattest parts of
    spheroid i: on the symmetry axis beyond both poles, and in the equatorial
    plane beyond the rim at n_side angles (exact distance d in both places,
    where the outward normal is along the offset).  Returns (T, 3); points
    inside another spheroid are dropped."""
    R = _quat_to_matrix(s.quat)
    pts = []
    for d in distances:
        pts.append(np.array([[0.0, 0.0, s.C[i] + d], [0.0, 0.0, -(s.C[i] + d)]]))
        ang = 2 * math.pi * (np.arange(n_side) + 0.25) / n_side
        r = s.A[i] + d
        pts.append(np.stack([r * np.cos(ang), r * np.sin(ang), np.zeros(n_side)], -1))
    X = np.concatenate(pts) @ R[i].T + s.center[i]
    keep = np.ones(len(X), bool)
    for j in range(s.M):
        if j == i:
            continue
        xl = (X - s.center[j]) @ R[j]
        f = (xl[:, 0] ** 2 + xl[:, 1] ** 2) / s.A[j] ** 2 + xl[:, 2] ** 2 / s.C[j] ** 2
        keep &= f > 1.0 + 1e-9
    return np.ascontiguousarray(X[keep])


def _quat_mul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Hamilton product a b of (w, x, y, z) quaternions (b may be (M, 4))."""
    aw, ax, ay, az = a
    bw, bx, by, bz = b[..., 0], b[..., 1], b[..., 2], b[..., 3]
    return np.stack([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw], axis=-1)


def rigid_motion(s: Suspension, seed: int, shift: float = 10.0) -> Suspension:
    """The same suspension moved as a whole by a seeded random rotation (about
    its centroid) and translation (U(-shift, shift)^3): a new geometry with
    the same gaps and shapes, used to give every request of a served stream
    its own geometry without a fresh placement."""
    rng = np.random.default_rng([seed, 161803])
    q = random_quaternions(rng, 1)[0]
    R = _quat_to_matrix(q[None])[0]
    c0 = s.center.mean(axis=0)
    center = (s.center - c0) @ R.T + c0 + rng.uniform(-shift, shift, 3)
    quat = _quat_mul(q, s.quat)
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    return Suspension(s.kind.copy(), s.A.copy(), s.C.copy(), center, quat, s.p, s.name)


def _serve_member(args):
    k, seed, M_range, p_choices, phi = args
    rng = np.random.default_rng([seed, k, 92821])
    M = int(round(math.exp(rng.uniform(math.log(M_range[0]), math.log(M_range[1])))))
    p = int(rng.choice(p_choices))
    return rsa_suspension(M, phi, 1000 + 97 * seed + k, p, name=f"serve{k}")


def serve_pool(n: int, seed: int = 0, M_range=(20, 500), p_choices=(8, 12, 16), phi: float = 0.20,
               workers: int = 1):
    """Suspensions for the served stream: M log-uniform in M_range, p from
    p_choices, shapes and placement as the 200-particle workload at volume
    fraction phi.  workers > 1 draws them in spawned processes (same
    result)."""
    jobs = [(k, seed, tuple(M_range), tuple(p_choices), phi) for k in range(n)]
    if workers <= 1:
        return [_serve_member(j) for j in jobs]
    import concurrent.futures as cf
    import multiprocessing as mp

    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_serve_member, jobs))
