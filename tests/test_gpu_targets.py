"""GPU parity of the particle-to-target evaluation (C ABI sbio_targets_* /
sbio_eval_targets, Sec. 4.1) against the CPU oracle: points on shells at
distances 10^-1 .. 10^-6 from every surface (the paper's shell tests) and
points spread through the suspension.  FP64 <= 1e-10 normwise vs the
oracle's method; mixed <= 1e-6 vs the GPU FP64 path."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


def gpu_eval(S, ts, sig, mu):
    sg = None if sig is None else torch.from_numpy(np.ascontiguousarray(sig)).cuda()
    mg = None if mu is None else torch.from_numpy(np.ascontiguousarray(mu)).cuda()
    So = None if sig is None else torch.full((ts.T,), float("nan"), dtype=torch.float64, device="cuda")
    Do = None if mu is None else torch.full((ts.T,), float("nan"), dtype=torch.float64, device="cuda")
    S.sbio_eval_targets(ts.h, sg, mg, So, Do)
    torch.cuda.synchronize()
    return (None if So is None else So.cpu().numpy()), (None if Do is None else Do.cpu().numpy())


@pytest.mark.parametrize("p", [2, 5, 8, 12, 16, 24])
def test_shell_points_fp64(S, ctx, p):
    s = I.rsa_suspension(5, 0.12, 700 + p, p, ar_range=(1.3, 4.0), name="t5")
    c = I.config_coefficients(s, p)
    X = I.shell_points(s, per_particle=3, seed=p, far_points=40)
    g = S.Geometry(ctx, s, near_factor=1.0)
    ts = S.TargetSet(g, X)
    og = OG.SuspensionGeom.from_suspension(s, near_factor=1.0)
    O = OL.LaplaceOracle(og)
    Sr, Dr = O.eval_points(X, c[0], c[1], "method")
    Sg, Dg = gpu_eval(S, ts, c[0], c[1])
    assert ts.n_near == int(og.point_near_matrix(X).sum())
    assert ts.n_far == O.point_far_pair_count(X)
    assert OL.normwise_rel_err(Sg, Sr) < TOL64
    assert OL.normwise_rel_err(Dg, Dr) < TOL64
    ts.close()
    g.close()


def test_mixed_vs_fp64_and_single_operators(S, ctx):
    s = I.config_suspension(3)
    c = I.config_coefficients(s, 2)
    X = I.shell_points(s, per_particle=2, seed=1, far_points=2000)
    g = S.Geometry(ctx, s, precision=S.SBIO_FP64)
    ts = S.TargetSet(g, X)
    S64, D64 = gpu_eval(S, ts, c[0], c[1])
    S1, _ = gpu_eval(S, ts, c[0], None)
    _, D1 = gpu_eval(S, ts, None, c[1])
    assert OL.normwise_rel_err(S1, S64) < 1e-13 and OL.normwise_rel_err(D1, D64) < 1e-13
    for tt in (2, -8):
        S.sbio_geom_set_precision(g.h, S.SBIO_MIXED)
        S.sbio_geom_set_launch_shape(g.h, tt, 0)
        Sm, Dm = gpu_eval(S, ts, c[0], c[1])
        assert OL.normwise_rel_err(Sm, S64) < TOLMIX and OL.normwise_rel_err(Dm, D64) < TOLMIX
    S.sbio_geom_set_launch_shape(g.h, 2, 0)
    S.sbio_geom_set_precision(g.h, S.SBIO_FP64)
    # sampled points against the oracle at this size
    og = OG.SuspensionGeom.from_suspension(s)
    sel = np.sort(np.random.default_rng(2).choice(len(X), 150, replace=False))
    Sr, Dr = OL.LaplaceOracle(og).eval_points(X[sel], c[0], c[1], "method")
    assert np.max(np.abs(S64[sel] - Sr)) / np.max(np.abs(S64)) < TOL64
    assert np.max(np.abs(D64[sel] - Dr)) / np.max(np.abs(D64)) < TOL64
    ts.close()
    g.close()


def test_points_at_nodes_give_exterior_limits(S, ctx):
    """At surface nodes the point path returns S and D+ = D + mu/2 of the
    on-surface apply (every pair near: near_factor large)."""
    s = I.rsa_suspension(3, 0.1, 41, 6)
    c = I.config_coefficients(s, 3)
    g = S.Geometry(ctx, s, near_factor=50.0)
    xyz, _, _ = S.sbio_geom_nodes(g.h)
    idx = np.arange(0, g.N, 5)
    ts = S.TargetSet(g, xyz[idx])
    Sp, Dp = gpu_eval(S, ts, c[0], c[1])
    sg, mg = torch.from_numpy(c[0]).cuda(), torch.from_numpy(c[1]).cuda()
    So = torch.empty(g.N, dtype=torch.float64, device="cuda")
    Do = torch.empty_like(So)
    S.sbio_apply_laplace(g.h, sg, mg, So, Do)
    torch.cuda.synchronize()
    og = OG.SuspensionGeom.from_suspension(s)
    mval = np.concatenate([OL.density_values(P, None, c[1][i])[1] for i, P in enumerate(og.parts)])
    assert OL.normwise_rel_err(Sp, So.cpu().numpy()[idx]) < 1e-11
    assert OL.normwise_rel_err(Dp, Do.cpu().numpy()[idx] + 0.5 * mval[idx]) < 1e-10
    ts.close()
    g.close()


def test_edge_cases(S, ctx):
    s = I.rsa_suspension(3, 0.1, 5, 4)
    g = S.Geometry(ctx, s)
    # empty set
    ts = S.TargetSet(g, np.zeros((0, 3)))
    assert ts.T == 0
    S.sbio_eval_targets(ts.h, torch.zeros(3 * 25, dtype=torch.float64, device="cuda"), None,
                        torch.zeros(1, dtype=torch.float64, device="cuda"), None)
    # the geometry refuses to go while a set is alive
    with pytest.raises(S.SbioError) as e:
        S.sbio_geom_destroy(g.h)
    assert e.value.code == S.SBIO_EINVAL
    ts.close()
    # a point inside a spheroid
    with pytest.raises(S.SbioError) as e:
        S.TargetSet(g, s.center[:1] + 1e-3)
    assert e.value.code == S.SBIO_EINVAL
    with pytest.raises(S.SbioError) as e:
        S.TargetSet(g, np.array([[np.nan, 0.0, 0.0]]))
    assert e.value.code == S.SBIO_EINVAL
    g.close()
