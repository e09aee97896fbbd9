"""GPU Stokes double layer (C ABI sbio_apply_stokes_dl,
sbio_eval_targets_stokes_dl) against the CPU oracle: FP64 <= 1e-10 normwise
at the nodes (principal value) and at points, rigid-body motions, and the
mixed path against FP64 (<= 1e-6)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import geometry as OG
from oracle import solve as OS
from oracle import stokes_dl as OSD
from paper_2506_20809_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL64 = 1e-10
TOLMIX = 1e-6


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as G

    G.build()
    import paper_2506_20809_gb300.sbio as S

    return S


@pytest.fixture(scope="module")
def ctx(S):
    return S.sbio_ctx_create(0, 0)


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def gpu_dl(S, g, q, precision=None):
    if precision is not None:
        S.sbio_geom_set_precision(g.h, precision)
    u = torch.full((g.N, 3), float("nan"), dtype=torch.float64, device="cuda")
    S.sbio_apply_stokes_dl(g.h, torch.from_numpy(np.ascontiguousarray(q)).cuda(), u)
    torch.cuda.synchronize()
    return u.cpu().numpy()


@pytest.mark.parametrize("p", [2, 5, 8, 12, 16, 20])
def test_cluster_fp64(S, ctx, p):
    s = I.rsa_suspension(3, 0.12, 900 + p, p, ar_range=(1.3, 4.0), name="dl3")
    q = np.random.default_rng(p).standard_normal((3, 3, (p + 1) ** 2)) / (1 + np.arange((p + 1) ** 2)) ** 0.5
    g = S.Geometry(ctx, s, near_factor=2.0)
    og = OG.SuspensionGeom.from_suspension(s, near_factor=2.0)
    Ur = OSD.StokesDLOracle(og).apply(q, "method")
    Ug = gpu_dl(S, g, q, S.SBIO_FP64)
    assert g.n_near > 0
    assert rel(Ug, Ur) < TOL64
    X = I.shell_points(s, distances=(1e-1, 1e-4), per_particle=2, seed=p, far_points=20)
    ts = S.TargetSet(g, X)
    u = torch.full((ts.T, 3), float("nan"), dtype=torch.float64, device="cuda")
    S.sbio_eval_targets_stokes_dl(ts.h, torch.from_numpy(q).cuda(), u)
    torch.cuda.synchronize()
    assert rel(u.cpu().numpy(), OSD.StokesDLOracle(og).eval_points(X, q, "method")) < TOL64
    ts.close()
    g.close()


def test_rigid_motion(S, ctx):
    """A rigid motion on one particle: -q/2 on its surface; at the other
    particles' nodes only the far quadrature's error of a zero field."""
    p = 10
    s = I.rsa_suspension(3, 0.1, 77, p)
    og = OG.SuspensionGeom.from_suspension(s)
    rng = np.random.default_rng(2)
    P = og.parts[1]
    vals = rng.standard_normal(3)[None, :] + np.cross(rng.standard_normal(3)[None, :], P.x - P.center)
    q = np.zeros((3, 3, (p + 1) ** 2))
    q[1] = np.stack([OS.analysis(P, vals[:, k]) for k in range(3)])
    g = S.Geometry(ctx, s)
    U = gpu_dl(S, g, q, S.SBIO_FP64)
    G = og.G
    assert np.max(np.abs(U[G:2 * G] + 0.5 * vals)) < 1e-11 * np.max(np.abs(vals))
    assert np.max(np.abs(np.delete(U, np.s_[G:2 * G], axis=0))) < 1e-6 * np.max(np.abs(vals))
    g.close()


def test_mixed_vs_fp64(S, ctx):
    s = I.config_suspension(3)
    p = s.p
    q = np.random.default_rng(4).standard_normal((s.M, 3, (p + 1) ** 2)) / (1 + np.arange((p + 1) ** 2))
    g = S.Geometry(ctx, s)
    U64 = gpu_dl(S, g, q, S.SBIO_FP64)
    Um = gpu_dl(S, g, q, S.SBIO_MIXED)
    print(f"stokes dl mixed vs fp64: {rel(Um, U64):.3e}")
    assert rel(Um, U64) < TOLMIX
    g.close()


@pytest.mark.parametrize("tt", [4, -2, -4, -8])
def test_mixed_far_forms(S, ctx, tt):
    """Scalar (4 targets per thread) and packed (2, 4, 8) stresslet far forms,
    with 0 (default) and 64 source splits, stay within the mixed bound of the
    FP64 path, at nodes and at points."""
    s = I.config_suspension(3)
    p = s.p
    q = np.random.default_rng(5).standard_normal((s.M, 3, (p + 1) ** 2)) / (1 + np.arange((p + 1) ** 2))
    g = S.Geometry(ctx, s)
    X = I.shell_points(s, per_particle=1, seed=3, far_points=2000)
    ts = S.TargetSet(g, X)
    qd = torch.from_numpy(q).cuda()
    U64 = gpu_dl(S, g, q, S.SBIO_FP64)
    P64 = torch.empty((ts.T, 3), dtype=torch.float64, device="cuda")
    S.sbio_eval_targets_stokes_dl(ts.h, qd, P64)
    torch.cuda.synchronize()
    P64 = P64.cpu().numpy()
    for splits in (0, 64):
        S.sbio_geom_set_stokes_tuning(g.h, tt, splits, 0)
        Um = gpu_dl(S, g, q, S.SBIO_MIXED)
        Pm = torch.full((ts.T, 3), float("nan"), dtype=torch.float64, device="cuda")
        S.sbio_eval_targets_stokes_dl(ts.h, qd, Pm)
        torch.cuda.synchronize()
        S.sbio_geom_set_precision(g.h, S.SBIO_FP64)
        assert rel(Um, U64) < TOLMIX, (tt, splits)
        assert rel(Pm.cpu().numpy(), P64) < TOLMIX, (tt, splits)
    ts.close()
    g.close()


def test_stokesdl100_sampled_against_oracle(S, ctx):
    """100 spheroids, p = 12 (the benchmark suspension): 30 sampled nodes of
    the FP64 GPU apply against the oracle's method, and the mixed apply within
    its bound of the same oracle values."""
    s = I.config_suspension(3)
    p = s.p
    q = np.random.default_rng(4).standard_normal((s.M, 3, (p + 1) ** 2)) / (1 + np.arange((p + 1) ** 2))
    g = S.Geometry(ctx, s)
    U64 = gpu_dl(S, g, q, S.SBIO_FP64)
    Um = gpu_dl(S, g, q, S.SBIO_MIXED)
    S.sbio_geom_set_precision(g.h, S.SBIO_FP64)
    og = OG.SuspensionGeom.from_suspension(s)
    tg = np.sort(np.random.default_rng(12).choice(g.N, 30, replace=False))
    Ur = OSD.StokesDLOracle(og).apply(q, "method", targets=tg)
    scale = np.max(np.abs(U64))
    assert np.max(np.abs(U64[tg] - Ur)) / scale < TOL64
    assert np.max(np.abs(Um[tg] - Ur)) / scale < TOLMIX
    g.close()


def test_limits_of_a_rigid_motion(S, ctx):
    """A rigid motion q on one particle: its exterior limit is 0 and its
    interior limit -q on that particle's surface (the field is 0 outside and
    -q inside); at the other particles' nodes all sides agree."""
    p = 10
    s = I.rsa_suspension(3, 0.1, 77, p)
    og = OG.SuspensionGeom.from_suspension(s)
    rng = np.random.default_rng(5)
    P = og.parts[1]
    vals = rng.standard_normal(3)[None, :] + np.cross(rng.standard_normal(3)[None, :], P.x - P.center)
    q = np.zeros((3, 3, (p + 1) ** 2))
    q[1] = np.stack([OS.analysis(P, vals[:, k]) for k in range(3)])
    g = S.Geometry(ctx, s, precision=S.SBIO_FP64)
    qd = torch.from_numpy(q).cuda()
    out = {}
    for side in (0, 1, -1):
        u = torch.full((g.N, 3), float("nan"), dtype=torch.float64, device="cuda")
        S.sbio_apply_stokes_dl_limit(g.h, qd, u, side)
        torch.cuda.synchronize()
        out[side] = u.cpu().numpy()
    G = og.G
    scale = np.max(np.abs(vals))
    assert np.max(np.abs(out[1][G:2 * G])) < 1e-11 * scale
    assert np.max(np.abs(out[-1][G:2 * G] + vals)) < 1e-11 * scale
    assert np.max(np.abs(out[0][G:2 * G] + 0.5 * vals)) < 1e-11 * scale
    rest = np.r_[0:G, 2 * G:3 * G]
    assert np.max(np.abs(out[1][rest] - out[0][rest])) <= 1e-14 * scale
    assert np.max(np.abs(out[-1][rest] - out[0][rest])) <= 1e-14 * scale
    with pytest.raises(S.SbioError) as e:
        S.sbio_apply_stokes_dl_limit(g.h, qd, torch.zeros((g.N, 3), dtype=torch.float64, device="cuda"), 3)
    assert e.value.code == S.SBIO_EINVAL
    g.close()


def test_points_forked_equals_in_order(S, ctx):
    """The point evaluation with the near pairs forked beside the far field
    (overlap on, the default) and with every phase in order on one stream
    (overlap off) agree to rounding: only the order of the atomic adds
    differs."""
    s = I.config_suspension(3)
    p = s.p
    q = np.random.default_rng(9).standard_normal((s.M, 3, (p + 1) ** 2)) / (1 + np.arange((p + 1) ** 2))
    qd = torch.from_numpy(q).cuda()
    out = {}
    for prec in (S.SBIO_FP64, S.SBIO_MIXED):
        g = S.Geometry(ctx, s, precision=prec)
        X = I.shell_points(s, per_particle=1, seed=6, far_points=2000)
        ts = S.TargetSet(g, X)
        for on in (1, 0):
            S.sbio_geom_set_overlap(g.h, on)
            u = torch.full((ts.T, 3), float("nan"), dtype=torch.float64, device="cuda")
            S.sbio_eval_targets_stokes_dl(ts.h, qd, u)
            torch.cuda.synchronize()
            out[on] = u.cpu().numpy()
        assert ts.n_near > 0
        assert rel(out[1], out[0]) < 1e-13, prec
        ts.close()
        g.close()
