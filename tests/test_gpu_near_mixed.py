"""The near field of SBIO_MIXED geometries (the FP32-contraction form: Q and
the coordinates in FP64, rho = extS q rounded to FP32, normalised Ferrers
recurrence and compensated n sums in FP32, m sums in FP64) against the plain
FP64 near field of the same geometry, part by part, at every order offered,
and the whole mixed apply against the oracle's method on sampled targets."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import geometry as OG
from oracle import laplace as OL
from paper_2506_20809_gb300 import inputs as I

pytestmark = pytest.mark.gpu
# stated bound of the mixed near part against the FP64 near part (normwise);
# an emulation of the form in NumPy put it at 1.3e-7 on 200 spheroids, p = 16
TOL_NEAR = 5e-7
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


def _parts(S, g, c, parts, prec):
    S.sbio_geom_set_precision(g.h, prec)
    sig = torch.from_numpy(np.ascontiguousarray(c[0])).cuda()
    mu = torch.from_numpy(np.ascontiguousarray(c[1])).cuda()
    So = torch.full((g.N,), float("nan"), dtype=torch.float64, device="cuda")
    Do = torch.full_like(So, float("nan"))
    S.sbio_apply_laplace_parts(g.h, sig, mu, So, Do, parts)
    torch.cuda.synchronize()
    return So.cpu().numpy(), Do.cpu().numpy()


@pytest.mark.parametrize("p", [1, 4, 8, 12, 16, 20, 24])
def test_mixed_near_part_matches_fp64(S, ctx, p):
    s = I.rsa_suspension(24, 0.25, 80 + p, p, name="nearmix")
    c = I.config_coefficients(s, p)
    g = S.Geometry(ctx, s, precision=S.SBIO_FP64)
    assert g.n_near > 0
    Sn64, Dn64 = _parts(S, g, c, S.SBIO_PART_NEAR, S.SBIO_FP64)
    Snm, Dnm = _parts(S, g, c, S.SBIO_PART_NEAR, S.SBIO_MIXED)
    eS, eD = OL.normwise_rel_err(Snm, Sn64), OL.normwise_rel_err(Dnm, Dn64)
    print(f"p={p}: near part mixed vs FP64 S {eS:.2e} D {eD:.2e}")
    assert eS < TOL_NEAR and eD < TOL_NEAR
    # single operators take the same form
    S.sbio_geom_set_precision(g.h, S.SBIO_MIXED)
    sig = torch.from_numpy(np.ascontiguousarray(c[0])).cuda()
    So = torch.full((g.N,), float("nan"), dtype=torch.float64, device="cuda")
    S.sbio_apply_laplace_parts(g.h, sig, None, So, None, S.SBIO_PART_NEAR)
    torch.cuda.synchronize()
    assert OL.normwise_rel_err(So.cpu().numpy(), Snm) < 1e-12
    g.close()


@pytest.mark.parametrize("ar,kind", [(26, 0), (64, 0), (64, 1)])
def test_mixed_near_part_high_aspect(S, ctx, ar, kind):
    s = I.elongated_pair(ar, kind, 12)
    c = I.config_coefficients(s, 3)
    g = S.Geometry(ctx, s, precision=S.SBIO_FP64)
    Sn64, Dn64 = _parts(S, g, c, S.SBIO_PART_NEAR, S.SBIO_FP64)
    Snm, Dnm = _parts(S, g, c, S.SBIO_PART_NEAR, S.SBIO_MIXED)
    eS, eD = OL.normwise_rel_err(Snm, Sn64), OL.normwise_rel_err(Dnm, Dn64)
    print(f"AR {ar} kind {kind}: near part mixed vs FP64 S {eS:.2e} D {eD:.2e}")
    assert eS < TOL_NEAR and eD < TOL_NEAR
    g.close()


def test_mixed_apply_against_oracle_sampled(S, ctx):
    """The whole mixed apply (FP32 far sums, mixed near form) on a
    60-spheroid suspension of the 200-spheroid recipe against the oracle's
    method on sampled targets, weighted towards targets with near pairs."""
    s = I.rsa_suspension(60, 0.20, 91, 16, name="mix60")
    c = I.config_coefficients(s, 4)
    g = S.Geometry(ctx, s, precision=S.SBIO_MIXED)
    Sm, Dm = _parts(S, g, c, S.SBIO_PART_ALL, S.SBIO_MIXED)
    og = OG.SuspensionGeom.from_suspension(s)
    near_t, _ = S.sbio_geom_near_pairs(g.h)
    rng = np.random.default_rng(6)
    tg = np.unique(np.concatenate([rng.choice(np.unique(near_t), 30, replace=False), rng.choice(g.N, 10)]))
    Sr, Dr = OL.LaplaceOracle(og).apply(c[0], c[1], "method", targets=tg)
    eS = np.max(np.abs(Sm[tg] - Sr)) / np.max(np.abs(Sr))
    eD = np.max(np.abs(Dm[tg] - Dr)) / np.max(np.abs(Dr))
    print(f"mixed apply vs oracle on {len(tg)} targets: S {eS:.2e} D {eD:.2e}")
    assert eS < TOLMIX and eD < TOLMIX
    g.close()
