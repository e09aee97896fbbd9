"""GPU Stokes single layer at arbitrary points (C ABI sbio_eval_targets_stokes):
velocity and pressure against the CPU oracle (FP64 <= 1e-10 normwise), the
mixed path against FP64 (<= 1e-6), and the on-surface apply at the nodes
(the single layer's velocity is continuous across the surface)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import geometry as OG
from oracle import stokes as OSK
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


def gpu_points(S, ts, f, pressure=True):
    fd = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    u = torch.full((ts.T, 3), float("nan"), dtype=torch.float64, device="cuda")
    pr = torch.full((ts.T,), float("nan"), dtype=torch.float64, device="cuda") if pressure else None
    S.sbio_eval_targets_stokes(ts.h, fd, u, pr)
    torch.cuda.synchronize()
    return u.cpu().numpy(), (pr.cpu().numpy() if pressure else None)


@pytest.mark.parametrize("p", [3, 8, 12, 16, 20])
def test_points_fp64(S, ctx, p):
    s = I.rsa_suspension(4, 0.12, 800 + p, p, ar_range=(1.3, 4.0), name="sp4")
    f = I.config_coefficients(s, p, ndens=3).transpose(1, 0, 2).copy()
    X = I.shell_points(s, distances=(1e-1, 1e-3, 1e-6), per_particle=3, seed=p, far_points=30)
    g = S.Geometry(ctx, s, near_factor=1.5)
    ts = S.TargetSet(g, X)
    og = OG.SuspensionGeom.from_suspension(s, near_factor=1.5)
    Ur, Pr = OSK.StokesOracle(og).eval_points(X, f, "method")
    Ug, Pg = gpu_points(S, ts, f)
    assert ts.n_near > 0
    assert rel(Ug, Ur) < TOL64
    assert rel(Pg, Pr) < TOL64
    Uv, _ = gpu_points(S, ts, f, pressure=False)
    assert rel(Uv, Ug) < 1e-13
    ts.close()
    g.close()


def test_mixed_and_nodes(S, ctx):
    s = I.config_suspension(3)
    f = I.config_coefficients(s, 4, ndens=3).transpose(1, 0, 2).copy()
    g = S.Geometry(ctx, s)
    X = I.shell_points(s, per_particle=2, seed=9, far_points=3000)
    ts = S.TargetSet(g, X)
    U64, P64 = gpu_points(S, ts, f)
    S.sbio_geom_set_precision(g.h, S.SBIO_MIXED)
    Um, Pm = gpu_points(S, ts, f)
    S.sbio_geom_set_precision(g.h, S.SBIO_FP64)
    print(f"stokes points mixed vs fp64: u {rel(Um, U64):.3e} p {rel(Pm, P64):.3e}")
    assert rel(Um, U64) < TOLMIX and rel(Pm, P64) < TOLMIX
    ts.close()
    # at a subset of the nodes: the on-surface apply (velocity is continuous)
    xyz, _, _ = S.sbio_geom_nodes(g.h)
    idx = np.arange(0, g.N, 97)
    ts = S.TargetSet(g, xyz[idx])
    Un, _ = gpu_points(S, ts, f, pressure=False)
    u = torch.empty((g.N, 3), dtype=torch.float64, device="cuda")
    S.sbio_apply_stokes_sl(g.h, torch.from_numpy(f).cuda(), u)
    torch.cuda.synchronize()
    assert rel(Un, u.cpu().numpy()[idx]) < 1e-9
    ts.close()
    g.close()


def test_rejects_high_order(S, ctx):
    s = I.rsa_suspension(2, 0.1, 4, 22)
    g = S.Geometry(ctx, s)
    ts = S.TargetSet(g, s.center + 5.0)
    f = torch.zeros((2, 3, 23 * 23), dtype=torch.float64, device="cuda")
    u = torch.zeros((2, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(S.SbioError) as e:
        S.sbio_eval_targets_stokes(ts.h, f, u, None)
    assert e.value.code == S.SBIO_ENOTSUP
    ts.close()
    g.close()


@pytest.mark.parametrize("tt", [1, 4, -2, -4, -8])
def test_far_forms_with_pressure(S, ctx, tt):
    """Every Stokeslet far form, which in mixed precision also sums the
    pressure in the same pass, stays within the mixed bound of FP64 for the
    velocity and the pressure."""
    s = I.config_suspension(3)
    f = I.config_coefficients(s, 6, ndens=3).transpose(1, 0, 2).copy()
    g = S.Geometry(ctx, s)
    X = I.shell_points(s, per_particle=1, seed=11, far_points=2500)
    ts = S.TargetSet(g, X)
    U64, P64 = gpu_points(S, ts, f)
    for splits in (0, 96):
        S.sbio_geom_set_stokes_tuning(g.h, tt, splits, 0)
        S.sbio_geom_set_precision(g.h, S.SBIO_MIXED)
        Um, Pm = gpu_points(S, ts, f)
        Uv, _ = gpu_points(S, ts, f, pressure=False)
        S.sbio_geom_set_precision(g.h, S.SBIO_FP64)
        assert rel(Um, U64) < TOLMIX and rel(Pm, P64) < TOLMIX, (tt, splits)
        assert rel(Uv, Um) < 1e-6, (tt, splits)
    ts.close()
    g.close()


def test_stokes100_points_sampled_against_oracle(S, ctx):
    """The benchmark suspension (100 spheroids, p = 12) at shell and box
    points: 40 sampled points of the FP64 GPU evaluation (velocity and
    pressure) against the oracle's method."""
    s = I.config_suspension(3)
    f = I.config_coefficients(s, 6, ndens=3).transpose(1, 0, 2).copy()
    g = S.Geometry(ctx, s)
    X = I.shell_points(s, per_particle=1, seed=4, far_points=2000)
    ts = S.TargetSet(g, X)
    U64, P64 = gpu_points(S, ts, f)
    og = OG.SuspensionGeom.from_suspension(s)
    sel = np.sort(np.random.default_rng(3).choice(len(X), 40, replace=False))
    Ur, Pr = OSK.StokesOracle(og).eval_points(X[sel], f, "method")
    assert np.max(np.abs(U64[sel] - Ur)) / np.max(np.abs(U64)) < TOL64
    assert np.max(np.abs(P64[sel] - Pr)) / np.max(np.abs(P64)) < TOL64
    ts.close()
    g.close()
