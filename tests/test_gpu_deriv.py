"""GPU parity of the normal-derivative operators S' and D' (C ABI
sbio_apply_laplace_deriv) against the CPU oracle (Theorem 3, eq.
(dSLevalformula)): FP64 <= 1e-10 normwise vs the oracle's method; mixed
(FP32 compensated far field) <= 1e-6 vs the GPU FP64 path."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import deriv as OD
from oracle import geometry as OG
from oracle import laplace as OL
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


def gpu_deriv(S, geom, sig, mu, precision=None):
    if precision is not None:
        S.sbio_geom_set_precision(geom.h, precision)
    sg = None if sig is None else torch.from_numpy(np.ascontiguousarray(sig)).cuda()
    mg = None if mu is None else torch.from_numpy(np.ascontiguousarray(mu)).cuda()
    Sp = None if sig is None else torch.full((geom.N,), float("nan"), dtype=torch.float64, device="cuda")
    Dp = None if mu is None else torch.full((geom.N,), float("nan"), dtype=torch.float64, device="cuda")
    S.sbio_apply_laplace_deriv(geom.h, sg, mg, Sp, Dp)
    torch.cuda.synchronize()
    return (None if Sp is None else Sp.cpu().numpy()), (None if Dp is None else Dp.cpu().numpy())


@pytest.mark.parametrize("p", [1, 3, 6, 9, 12, 16, 20])
def test_cluster_fp64(S, ctx, p):
    """Several spheroids of both kinds close enough for near pairs (near
    factor 2): self + near gradients + far quadrature, every order p."""
    s = I.rsa_suspension(4, 0.12, 600 + p, p, ar_range=(1.3, 4.0), name="d4")
    c = I.config_coefficients(s, p)
    g = S.Geometry(ctx, s, near_factor=2.0)
    og = OG.SuspensionGeom.from_suspension(s, near_factor=2.0)
    Spr, Dpr = OD.DerivOracle(og).apply(c[0], c[1], "method")
    Spg, Dpg = gpu_deriv(S, g, c[0], c[1], S.SBIO_FP64)
    assert g.n_near > 0
    assert OL.normwise_rel_err(Spg, Spr) < TOL64
    assert OL.normwise_rel_err(Dpg, Dpr) < TOL64
    # one operator at a time gives the same numbers (up to the order of the
    # atomic accumulation)
    Sp1, _ = gpu_deriv(S, g, c[0], None)
    _, Dp1 = gpu_deriv(S, g, None, c[1])
    assert OL.normwise_rel_err(Sp1, Spg) < 1e-13 and OL.normwise_rel_err(Dp1, Dpg) < 1e-13
    g.close()


def test_conductor_field(S, ctx):
    """One spheroid with the equilibrium density: S' = -sigma/2 at every node."""
    s = I.Suspension(np.array([1], np.int32), np.array([1.3]), np.array([0.6]), np.zeros((1, 3)),
                     np.array([[0.9, 0.2, -0.3, 0.25]]) / np.linalg.norm([0.9, 0.2, -0.3, 0.25]), 10)
    sig = np.zeros((1, 121))
    sig[0, 0] = 1.0
    g = S.Geometry(ctx, s)
    og = OG.SuspensionGeom.from_suspension(s)
    sval, _ = OL.density_values(og.parts[0], sig[0], None)
    Sp, _ = gpu_deriv(S, g, sig, None, S.SBIO_FP64)
    assert np.max(np.abs(Sp + 0.5 * sval)) < 1e-12 * np.max(np.abs(sval))
    g.close()


@pytest.fixture(scope="module")
def stokes100(S, ctx):
    s = I.config_suspension(3)
    c = I.config_coefficients(s, 1)
    g = S.Geometry(ctx, s)
    yield s, c, g
    g.close()


def test_mixed_vs_fp64(S, stokes100):
    s, c, g = stokes100
    Sp64, Dp64 = gpu_deriv(S, g, c[0], c[1], S.SBIO_FP64)
    Spm, Dpm = gpu_deriv(S, g, c[0], c[1], S.SBIO_MIXED)
    S.sbio_geom_set_precision(g.h, S.SBIO_FP64)
    eS, eD = OL.normwise_rel_err(Spm, Sp64), OL.normwise_rel_err(Dpm, Dp64)
    print(f"deriv mixed vs fp64: S' {eS:.3e} D' {eD:.3e}")
    assert eS < TOLMIX and eD < TOLMIX


@pytest.mark.parametrize("tt", [2, -8])
def test_mixed_far_forms(S, stokes100, tt):
    """Scalar (tt > 0) and packed f32x2 (tt < 0) forms of the mixed far
    kernel stay within the mixed bound of the FP64 path."""
    s, c, g = stokes100
    Sp64, Dp64 = gpu_deriv(S, g, c[0], c[1], S.SBIO_FP64)
    saved = S.sbio_geom_get_tuning(g.h)
    try:
        S.sbio_geom_set_launch_shape(g.h, tt, 0)
        Spm, Dpm = gpu_deriv(S, g, c[0], c[1], S.SBIO_MIXED)
    finally:
        S.sbio_geom_set_launch_shape(g.h, saved["far_tt"], saved["far_splits"])
        S.sbio_geom_set_precision(g.h, S.SBIO_FP64)
    assert OL.normwise_rel_err(Spm, Sp64) < TOLMIX and OL.normwise_rel_err(Dpm, Dp64) < TOLMIX


def test_sampled_against_oracle(S, stokes100):
    """100 spheroids, p = 12: sampled nodes against the oracle's method."""
    s, c, g = stokes100
    Spg, Dpg = gpu_deriv(S, g, c[0], c[1], S.SBIO_FP64)
    og = OG.SuspensionGeom.from_suspension(s)
    tg = np.sort(np.random.default_rng(11).choice(g.N, 120, replace=False))
    Spr, Dpr = OD.DerivOracle(og).apply(c[0], c[1], "method", targets=tg)
    assert np.max(np.abs(Spg[tg] - Spr)) / np.max(np.abs(Spg)) < TOL64
    assert np.max(np.abs(Dpg[tg] - Dpr)) / np.max(np.abs(Dpg)) < TOL64


def test_invalid_arguments(S, ctx):
    s = I.rsa_suspension(2, 0.1, 3, 22)
    g = S.Geometry(ctx, s)
    c = I.config_coefficients(s, 0)
    with pytest.raises(S.SbioError) as e:
        gpu_deriv(S, g, c[0], c[1])
    assert e.value.code == S.SBIO_ENOTSUP
    g.close()
    s = I.rsa_suspension(2, 0.1, 3, 4)
    g = S.Geometry(ctx, s)
    x = torch.zeros(2 * 25, dtype=torch.float64, device="cuda")
    out = torch.zeros(g.N, dtype=torch.float64, device="cuda")
    with pytest.raises(S.SbioError) as e:
        S.sbio_apply_laplace_deriv(g.h, x, None, None, out)
    assert e.value.code == S.SBIO_EINVAL
    g.close()


def gpu_point_deriv(S, ts, dirs, sig, mu):
    dd = torch.from_numpy(np.ascontiguousarray(dirs)).cuda()
    sg = None if sig is None else torch.from_numpy(np.ascontiguousarray(sig)).cuda()
    mg = None if mu is None else torch.from_numpy(np.ascontiguousarray(mu)).cuda()
    So = None if sig is None else torch.full((ts.T,), float("nan"), dtype=torch.float64, device="cuda")
    Do = None if mu is None else torch.full((ts.T,), float("nan"), dtype=torch.float64, device="cuda")
    S.sbio_eval_targets_deriv(ts.h, dd, sg, mg, So, Do)
    torch.cuda.synchronize()
    return (None if So is None else So.cpu().numpy()), (None if Do is None else Do.cpu().numpy())


def unit_dirs(n, seed):
    v = np.random.default_rng(seed).standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


@pytest.mark.parametrize("p", [2, 7, 12, 16, 20])
def test_points_fp64(S, ctx, p):
    """Shell points 1e-1 .. 1e-6 outside every surface plus spread points,
    random unit directions: against the oracle's point method."""
    s = I.rsa_suspension(4, 0.12, 900 + p, p, ar_range=(1.3, 4.0), name="dp4")
    c = I.config_coefficients(s, p)
    X = I.shell_points(s, distances=(1e-1, 1e-3, 1e-6), per_particle=3, seed=p, far_points=30)
    E = unit_dirs(len(X), p)
    g = S.Geometry(ctx, s, near_factor=1.5)
    ts = S.TargetSet(g, X)
    og = OG.SuspensionGeom.from_suspension(s, near_factor=1.5)
    Sr, Dr = OD.DerivOracle(og).eval_points(X, E, c[0], c[1], "method")
    Sg, Dg = gpu_point_deriv(S, ts, E, c[0], c[1])
    assert ts.n_near > 0
    assert OL.normwise_rel_err(Sg, Sr) < TOL64
    assert OL.normwise_rel_err(Dg, Dr) < TOL64
    S1, _ = gpu_point_deriv(S, ts, E, c[0], None)
    _, D1 = gpu_point_deriv(S, ts, E, None, c[1])
    assert OL.normwise_rel_err(S1, Sg) < 1e-13 and OL.normwise_rel_err(D1, Dg) < 1e-13
    ts.close()
    g.close()


def test_points_mixed_forms_and_linearity(S, stokes100):
    """Mixed scalar and packed far forms within the mixed bound of FP64 at
    3000 spread points; the result is linear in the direction."""
    s, c, g = stokes100
    X = I.shell_points(s, per_particle=1, seed=4, far_points=3000)
    E = unit_dirs(len(X), 5)
    ts = S.TargetSet(g, X)
    S.sbio_geom_set_precision(g.h, S.SBIO_FP64)
    S64, D64 = gpu_point_deriv(S, ts, E, c[0], c[1])
    S3, D3 = gpu_point_deriv(S, ts, -3.0 * E, c[0], c[1])
    assert OL.normwise_rel_err(S3, -3.0 * S64) < 1e-13 and OL.normwise_rel_err(D3, -3.0 * D64) < 1e-13
    saved = S.sbio_geom_get_tuning(g.h)
    try:
        S.sbio_geom_set_precision(g.h, S.SBIO_MIXED)
        for tt in (2, -8):
            S.sbio_geom_set_launch_shape(g.h, tt, 0)
            Sm, Dm = gpu_point_deriv(S, ts, E, c[0], c[1])
            assert OL.normwise_rel_err(Sm, S64) < TOLMIX and OL.normwise_rel_err(Dm, D64) < TOLMIX
    finally:
        S.sbio_geom_set_launch_shape(g.h, saved["far_tt"], saved["far_splits"])
        S.sbio_geom_set_precision(g.h, S.SBIO_FP64)
    og = OG.SuspensionGeom.from_suspension(s)
    sel = np.sort(np.random.default_rng(6).choice(len(X), 100, replace=False))
    Sr, Dr = OD.DerivOracle(og).eval_points(X[sel], E[sel], c[0], c[1], "method")
    assert np.max(np.abs(S64[sel] - Sr)) / np.max(np.abs(S64)) < TOL64
    assert np.max(np.abs(D64[sel] - Dr)) / np.max(np.abs(D64)) < TOL64
    ts.close()


def test_points_at_nodes_give_exterior_limits(S, ctx):
    """At surface nodes along the outward normals (every pair near): the
    exterior limits S'+ = S' - sigma/2 and D' of the on-surface apply."""
    s = I.rsa_suspension(3, 0.1, 43, 7)
    c = I.config_coefficients(s, 7)
    g = S.Geometry(ctx, s, near_factor=50.0)
    xyz, nrm, _ = S.sbio_geom_nodes(g.h)
    idx = np.arange(0, g.N, 5)
    ts = S.TargetSet(g, xyz[idx])
    Spt, Dpt = gpu_point_deriv(S, ts, nrm[idx], c[0], c[1])
    Sp, Dp = gpu_deriv(S, g, c[0], c[1], S.SBIO_FP64)
    og = OG.SuspensionGeom.from_suspension(s)
    sval = np.concatenate([OL.density_values(P, c[0][i], None)[0] for i, P in enumerate(og.parts)])
    assert OL.normwise_rel_err(Spt, Sp[idx] - 0.5 * sval[idx]) < 1e-10
    assert OL.normwise_rel_err(Dpt, Dp[idx]) < 1e-9
    ts.close()
    g.close()


def test_points_invalid_arguments(S, ctx):
    s = I.rsa_suspension(2, 0.1, 3, 4)
    g = S.Geometry(ctx, s)
    ts = S.TargetSet(g, s.center + 5.0)
    x = torch.zeros(2 * 25, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    dirs = torch.zeros((2, 3), dtype=torch.float64, device="cuda")
    for args in ((None, x, None, out, None), (dirs, x, None, None, out), (dirs, None, None, None, None)):
        with pytest.raises(S.SbioError) as e:
            S.sbio_eval_targets_deriv(ts.h, *args)
        assert e.value.code == S.SBIO_EINVAL
    ts.close()
    # an empty set: nothing to do, no direction array needed
    ts = S.TargetSet(g, np.zeros((0, 3)))
    S.sbio_eval_targets_deriv(ts.h, None, x, None, out, None)
    ts.close()
    g.close()
