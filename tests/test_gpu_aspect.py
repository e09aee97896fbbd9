"""Near-field accuracy at high aspect ratio (the paper's stress tests run
prolate spheroids up to aspect ratio 64).  Close to a slender prolate's side
or a thin oblate's faces the radial coordinate u approaches u0 = 1 + O(1/R^2)
(prolate) or 0 (oblate), where the backward recurrence for Q_n^m has to start
~19/atanh(1/R) steps above the top order.  Every GPU near kernel (S and D,
S' and D', the Stokes single layer) must still match the oracle at the
1e-10 bar, at nodes and at points 1e-3 from the poles and the rim; aspect
ratios beyond the supported bound are refused."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import deriv as OD
from oracle import geometry as OG
from oracle import laplace as OL
from oracle import stokes as OS
from paper_2506_20809_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL64 = 1e-10
TOLMIX = 1e-6
CASES = [(ar, kind) for ar in (10, 26, 64) for kind in (0, 1)]


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


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _nan(*shape):
    return torch.full(shape, float("nan"), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("ar,kind", CASES)
def test_laplace_nodes_and_points(S, ctx, ar, kind):
    s = I.elongated_pair(ar, kind, 12)
    c = I.config_coefficients(s, 3)
    og = OG.SuspensionGeom.from_suspension(s)
    O = OL.LaplaceOracle(og)
    Sr, Dr = O.apply(c[0], c[1], "method")
    X = np.concatenate([I.extreme_points(s, 0, (1e-1, 1e-2, 1e-3)),
                        I.shell_points(s, distances=(1e-3,), per_particle=16, seed=ar)])
    SXr, DXr = O.eval_points(X, c[0], c[1], "method")
    out = {}
    for prec in ("fp64", "mixed"):
        g = S.Geometry(ctx, s, precision=S.SBIO_FP64 if prec == "fp64" else S.SBIO_MIXED)
        assert g.n_near > 0
        So, Do = _nan(g.N), _nan(g.N)
        S.sbio_apply_laplace(g.h, _cuda(c[0]), _cuda(c[1]), So, Do)
        ts = S.TargetSet(g, X)
        assert ts.n_near > 0
        SX, DX = _nan(ts.T), _nan(ts.T)
        S.sbio_eval_targets(ts.h, _cuda(c[0]), _cuda(c[1]), SX, DX)
        torch.cuda.synchronize()
        out[prec] = [t.cpu().numpy() for t in (So, Do, SX, DX)]
        ts.close()
        g.close()
    for got, ref in zip(out["fp64"], (Sr, Dr, SXr, DXr)):
        assert OL.normwise_rel_err(got, ref) < TOL64, (ar, kind)
    for got, ref in zip(out["mixed"], out["fp64"]):
        assert OL.normwise_rel_err(got, ref) < TOLMIX, (ar, kind)


@pytest.mark.parametrize("ar,kind", [(26, 0), (64, 0), (64, 1)])
def test_derivatives_and_stokes(S, ctx, ar, kind):
    """The gradient kernels (S' and D' at nodes, the Stokes single layer)
    share the Miller start with the value kernels."""
    s = I.elongated_pair(ar, kind, 10)
    c = I.config_coefficients(s, 4)
    f = I.config_coefficients(s, 5, ndens=3).transpose(1, 0, 2)
    og = OG.SuspensionGeom.from_suspension(s)
    Spr, Dpr = OD.DerivOracle(og).apply(c[0], c[1], "method")
    Ur = OS.StokesOracle(og).apply(f, "method")
    g = S.Geometry(ctx, s, precision=S.SBIO_FP64)
    Sp, Dp = _nan(g.N), _nan(g.N)
    S.sbio_apply_laplace_deriv(g.h, _cuda(c[0]), _cuda(c[1]), Sp, Dp)
    u = _nan(g.N, 3)
    S.sbio_apply_stokes_sl(g.h, _cuda(f), u)
    torch.cuda.synchronize()
    assert OL.normwise_rel_err(Sp.cpu().numpy(), Spr) < TOL64
    assert OL.normwise_rel_err(Dp.cpu().numpy(), Dpr) < TOL64
    assert OL.normwise_rel_err(u.cpu().numpy(), Ur) < TOL64
    g.close()


def test_aspect_ratio_beyond_bound_is_refused(S, ctx):
    s = I.elongated_pair(5000, 0, 6)
    with pytest.raises(S.SbioError) as e:
        S.Geometry(ctx, s)
    assert e.value.code == S.SBIO_EINVAL
    assert "aspect ratio" in str(e.value)
