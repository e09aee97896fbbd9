"""GPU parity of the Stokes single layer (C ABI) against the CPU oracle
(Sec. 4.3, eq. (stokes)): FP64 <= 1e-10 normwise vs the oracle's method
(near/self through Laplace expansions, Stokeslet far quadrature); mixed
(FP32 compensated Stokeslet far field) <= 1e-6 vs the GPU FP64 path."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import geometry as OG
from oracle import stokes as OS
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


def relerr(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def gpu_stokes(S, geom, f, precision=None):
    if precision is not None:
        S.sbio_geom_set_precision(geom.h, precision)
    fg = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    u = torch.full((geom.N, 3), float("nan"), dtype=torch.float64, device="cuda")
    S.sbio_apply_stokes_sl(geom.h, fg, u)
    torch.cuda.synchronize()
    return u.cpu().numpy()


@pytest.mark.parametrize("p", [2, 5, 8, 12, 16, 20])
def test_cluster_fp64(S, ctx, p):
    s = I.rsa_suspension(3, 0.12, 200 + p, p, ar_range=(1.3, 4.0), name="c3")
    f = I.config_coefficients(s, p, ndens=3).transpose(1, 0, 2).copy()    # (M, 3, nc)
    g = S.Geometry(ctx, s, near_factor=2.0)
    og = OG.SuspensionGeom.from_suspension(s, near_factor=2.0)
    Ur = OS.StokesOracle(og).apply(f, "method")
    Ug = gpu_stokes(S, g, f, S.SBIO_FP64)
    assert g.n_near > 0
    assert relerr(Ug, Ur) < TOL64
    g.close()


def test_translating_spheroid_uniform_velocity(S, ctx):
    s = I.Suspension(np.array([0], np.int32), np.array([0.4]), np.array([1.5]), np.zeros((1, 3)),
                     np.array([[0.8, 0.1, 0.5, -0.3]]) / np.linalg.norm([0.8, 0.1, 0.5, -0.3]), 8)
    f = np.zeros((1, 3, 81))
    f[0, :, 0] = [0.3, -0.5, 0.8]
    g = S.Geometry(ctx, s)
    U = gpu_stokes(S, g, f, S.SBIO_FP64)
    assert np.max(np.ptp(U, axis=0)) < 1e-12 * np.max(np.abs(U))
    g.close()


@pytest.fixture(scope="module")
def stokes100(S, ctx):
    s = I.config_suspension(3)
    f = I.config_coefficients(s, 0, ndens=3).transpose(1, 0, 2).copy()
    g = S.Geometry(ctx, s)
    return s, f, g


def test_stokes100_sampled_fp64(S, stokes100):
    s, f, g = stokes100
    Ug = gpu_stokes(S, g, f, S.SBIO_FP64)
    og = OG.SuspensionGeom.from_suspension(s)
    tg = np.sort(np.random.default_rng(3).choice(g.N, 150, replace=False))
    Ur = OS.StokesOracle(og).apply(f, "method", targets=tg)
    assert np.max(np.abs(Ug[tg] - Ur)) / np.max(np.abs(Ug)) < TOL64


def test_stokes100_mixed_vs_fp64(S, stokes100):
    s, f, g = stokes100
    U64 = gpu_stokes(S, g, f, S.SBIO_FP64)
    Um = gpu_stokes(S, g, f, S.SBIO_MIXED)
    S.sbio_geom_set_precision(g.h, S.SBIO_FP64)
    e = relerr(Um, U64)
    print(f"stokes mixed vs fp64: {e:.3e}")
    assert e < TOLMIX


@pytest.mark.parametrize("tt,splits", [(1, 0), (4, 2), (8, 0), (-2, 0), (-4, 3), (-8, 0)])
def test_stokes_far_launch_shapes(S, stokes100, tt, splits):
    """Every far-field launch shape of the Stokeslet kernel stays within the
    mixed-precision bound of the FP64 path."""
    s, f, g = stokes100
    U64 = gpu_stokes(S, g, f, S.SBIO_FP64)
    saved = S.sbio_geom_get_stokes_tuning(g.h)
    try:
        S.sbio_geom_set_stokes_tuning(g.h, tt, splits, 1)
        Um = gpu_stokes(S, g, f, S.SBIO_MIXED)
    finally:
        S.sbio_geom_set_stokes_tuning(g.h, saved["far_tt"], saved["far_splits"], saved["near_ctas_per_sm"])
        S.sbio_geom_set_precision(g.h, S.SBIO_FP64)
    assert relerr(Um, U64) < TOLMIX


def test_stokes_autotune_and_host_entry(S, stokes100):
    """The Stokes autotuner picks a valid shape, leaves the Laplace settings
    alone, and the host entry point gives the device path's numbers."""
    s, f, g = stokes100
    S.sbio_geom_set_precision(g.h, S.SBIO_MIXED)
    lap = S.sbio_geom_get_tuning(g.h)
    try:
        tt, sp, ms = S.sbio_geom_autotune_stokes(g.h)
        assert tt in (1, 2, 4, 8, -2, -4, -8) and sp >= 1 and ms > 0
        assert S.sbio_geom_get_tuning(g.h) == lap
        assert S.sbio_geom_get_stokes_tuning(g.h)["far_tt"] == tt
        Ud = gpu_stokes(S, g, f)
        Uh = np.zeros((g.N, 3))
        S.sbio_apply_stokes_sl_host(g.h, np.ascontiguousarray(f), Uh)
        assert np.max(np.abs(Uh - Ud)) <= 1e-12 * np.max(np.abs(Ud))
    finally:
        S.sbio_geom_set_precision(g.h, S.SBIO_FP64)


def test_stokes_tuning_rejects_bad_values(S, stokes100):
    g = stokes100[2]
    for args in [(3, 0, 0), (2, -1, 0), (2, 0, -1)]:
        with pytest.raises(S.SbioError) as e:
            S.sbio_geom_set_stokes_tuning(g.h, *args)
        assert e.value.code == S.SBIO_EINVAL
