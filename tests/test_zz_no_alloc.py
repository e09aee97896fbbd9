"""The allocation-free self-interaction entry point (for callers whose device
memory belongs to someone else and who therefore must not cudaMalloc) gives
the same result as the self part of the regular apply, call after call.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2506_20809_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL64 = 1e-10


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as G

    G.build()
    import paper_2506_20809_gb300.sbio as S

    return S


def _relerr(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _regular_self(S, ctx, susp, sig, mu):
    g = S.Geometry(ctx, susp)
    So = torch.empty(g.N, dtype=torch.float64, device="cuda")
    Do = torch.empty_like(So)
    S.sbio_apply_laplace_parts(g.h, sig, mu, So, Do, S.SBIO_PART_SELF)
    torch.cuda.synchronize()
    out = So.cpu().numpy(), Do.cpu().numpy()
    g.close()
    return out


def test_noalloc_self_matches_regular_entry_point_twice(S):
    ctx = S.sbio_ctx_create(0, 0)
    cases = [(I.config_suspension(1), 0), (I.rsa_suspension(5, 0.1, 11, 12, name="five"), 1)]
    for susp, seed in cases:            # two calls in a row, different sizes and data
        coef = I.config_coefficients(susp, seed)
        sig = torch.from_numpy(coef[0]).cuda()
        mu = torch.from_numpy(coef[1]).cuda()
        Sr, Dr = _regular_self(S, ctx, susp, sig, mu)
        sph = S.make_spheroids(susp.kind, susp.A, susp.C, susp.center, susp.quat)
        So = torch.full((len(Sr),), float("nan"), dtype=torch.float64, device="cuda")
        Do = torch.full_like(So, float("nan"))
        S.sbio_apply_self_noalloc(sph, susp.p, sig, mu, So, Do)
        torch.cuda.synchronize()
        assert _relerr(So.cpu().numpy(), Sr) < TOL64
        assert _relerr(Do.cpu().numpy(), Dr) < TOL64
    S.sbio_ctx_destroy(ctx)


def test_noalloc_rejects_requests_beyond_the_fixed_array(S):
    base = I.config_suspension(1)
    susp = base.subset(np.arange(200) % 8)   # 200 spheroids at p = 16: far above 8 MiB
    susp.p = 16
    sph = S.make_spheroids(susp.kind, susp.A, susp.C, susp.center, susp.quat)
    nc = (susp.p + 1) ** 2
    sig = torch.zeros(susp.M * nc, dtype=torch.float64, device="cuda")
    out = torch.zeros(susp.M * (susp.p + 1) * 2 * (susp.p + 1), dtype=torch.float64, device="cuda")
    with pytest.raises(S.SbioError) as e:
        S.sbio_apply_self_noalloc(sph, susp.p, sig, None, out, None)
    assert e.value.code == S.SBIO_EINVAL
    assert "scratch" in str(e.value)


def test_noalloc_refuses_a_capturing_stream(S):
    # the tables are staged from a host buffer freed when the call returns,
    # so a call recorded into a graph would read freed memory at replay:
    # the entry point refuses a stream that is being captured
    susp = I.config_suspension(1)
    coef = I.config_coefficients(susp, 0)
    sig = torch.from_numpy(coef[0]).cuda()
    sph = S.make_spheroids(susp.kind, susp.A, susp.C, susp.center, susp.quat)
    out = torch.zeros(susp.M * (susp.p + 1) * 2 * (susp.p + 1), dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    x = torch.zeros(4, device="cuda")
    graph = torch.cuda.CUDAGraph()
    err = None
    torch.cuda.synchronize()
    with torch.cuda.graph(graph, stream=side):
        x.add_(1.0)                              # keeps the captured graph non-empty
        try:
            S.sbio_apply_self_noalloc(sph, susp.p, sig, None, out, None, stream=side.cuda_stream)
        except S.SbioError as e:
            err = e
    assert err is not None and err.code == S.SBIO_EINVAL
    assert "captured" in str(err)
    graph.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0
