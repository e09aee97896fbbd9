"""Batched apply (one graph, persistent far-field kernel over many suspensions)
against the single-geometry FP64 path, within the mixed-precision bound."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2506_20809_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOLMIX = 1e-6


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as G

    G.build()
    import paper_2506_20809_gb300.sbio as S

    return S


def relerr(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_batch_matches_single_geometry(S):
    ctx = S.sbio_ctx_create(0, 0)
    specs = [(3, 4), (7, 6), (12, 8), (5, 12), (20, 5), (9, 16)]
    susps = [I.rsa_suspension(M, 0.1, 300 + k, p, name=f"b{k}") for k, (M, p) in enumerate(specs)]
    geoms = [S.Geometry(ctx, s, precision=S.SBIO_MIXED) for s in susps]
    refs = []
    for s, g in zip(susps, geoms):
        c = I.config_coefficients(s, 5)
        sig, mu = torch.from_numpy(c[0]).cuda(), torch.from_numpy(c[1]).cuda()
        So = torch.empty(g.N, dtype=torch.float64, device="cuda")
        Do = torch.empty_like(So)
        S.sbio_geom_set_precision(g.h, S.SBIO_FP64)
        S.sbio_apply_laplace(g.h, sig, mu, So, Do)
        S.sbio_geom_set_precision(g.h, S.SBIO_MIXED)
        refs.append((sig, mu, So.clone(), Do.clone()))
    b = S.sbio_batch_create(ctx, geoms)
    info = S.sbio_batch_info(b)
    assert info["n_items"] > 0 and info["far_pairs"] == sum(g.n_far for g in geoms)
    outS = [torch.full((g.N,), float("nan"), dtype=torch.float64, device="cuda") for g in geoms]
    outD = [torch.full_like(o, float("nan")) for o in outS]
    for rep in range(2):                      # capture, then replay
        S.sbio_batch_apply(b, [r[0] for r in refs], [r[1] for r in refs], outS, outD)
        torch.cuda.synchronize()
        for k, r in enumerate(refs):
            assert relerr(outS[k].cpu().numpy(), r[2].cpu().numpy()) < TOLMIX
            assert relerr(outD[k].cpu().numpy(), r[3].cpu().numpy()) < TOLMIX
    # new values in the same buffers: the replay must see them
    for r in refs:
        r[0].mul_(-2.0)
    S.sbio_batch_apply(b, [r[0] for r in refs], [r[1] for r in refs], outS, outD)
    torch.cuda.synchronize()
    for k, r in enumerate(refs):
        assert relerr(outS[k].cpu().numpy(), -2.0 * r[2].cpu().numpy()) < TOLMIX
    # new output buffers: re-capture
    outS2 = [torch.empty_like(o) for o in outS]
    outD2 = [torch.empty_like(o) for o in outD]
    S.sbio_batch_set_far_tt(b, -4)
    S.sbio_batch_apply(b, [r[0] for r in refs], [r[1] for r in refs], outS2, outD2)
    torch.cuda.synchronize()
    for k, r in enumerate(refs):
        assert relerr(outD2[k].cpu().numpy(), r[3].cpu().numpy()) < TOLMIX
    S.sbio_batch_destroy(b)
    for g in geoms:
        g.close()
    S.sbio_ctx_destroy(ctx)


def test_batch_rejects_fp64_geometries(S):
    ctx = S.sbio_ctx_create(0, 0)
    s = I.rsa_suspension(3, 0.1, 7, 4)
    g = S.Geometry(ctx, s, precision=S.SBIO_FP64)
    with pytest.raises(S.SbioError) as e:
        S.sbio_batch_create(ctx, [g])
    assert e.value.code == S.SBIO_EINVAL
    g.close()
    S.sbio_ctx_destroy(ctx)


def test_batch_against_oracle_sampled(S):
    """Each suspension of one batched step against the CPU oracle's method on
    sampled targets, at the mixed bound; the batch spans the batched
    workload's ranges, including a suspension with M >= 300 and one at
    p = 20."""
    from oracle import geometry as OG
    from oracle import laplace as OL

    ctx = S.sbio_ctx_create(0, 0)
    specs = [(320, 20, 0.15), (40, 8, 0.25), (12, 12, 0.05), (90, 16, 0.20)]
    susps = [I.rsa_suspension(M, phi, 640 + k, p, name=f"bo{k}") for k, (M, p, phi) in enumerate(specs)]
    geoms = [S.Geometry(ctx, s, precision=S.SBIO_MIXED) for s in susps]
    coefs = [I.config_coefficients(s, 11 + k) for k, s in enumerate(susps)]
    sig = [torch.from_numpy(c[0]).cuda() for c in coefs]
    mu = [torch.from_numpy(c[1]).cuda() for c in coefs]
    outS = [torch.full((g.N,), float("nan"), dtype=torch.float64, device="cuda") for g in geoms]
    outD = [torch.full_like(o, float("nan")) for o in outS]
    b = S.sbio_batch_create(ctx, geoms)
    S.sbio_batch_apply(b, sig, mu, outS, outD)
    torch.cuda.synchronize()
    for k, (s, g, c) in enumerate(zip(susps, geoms, coefs)):
        og = OG.SuspensionGeom.from_suspension(s)
        tg = np.sort(np.random.default_rng(k).choice(g.N, 20, replace=False))
        Sr, Dr = OL.LaplaceOracle(og).apply(c[0], c[1], "method", targets=tg)
        eS = np.max(np.abs(outS[k].cpu().numpy()[tg] - Sr)) / np.max(np.abs(Sr))
        eD = np.max(np.abs(outD[k].cpu().numpy()[tg] - Dr)) / np.max(np.abs(Dr))
        print(f"batch suspension {k} (M={s.M}, p={s.p}): S {eS:.2e} D {eD:.2e}")
        assert eS < TOLMIX and eD < TOLMIX, (k, eS, eD)
    S.sbio_batch_destroy(b)
    for g in geoms:
        g.close()
    S.sbio_ctx_destroy(ctx)


def test_batch_autotune_in_library(S):
    """The library's batch autotuner picks a far shape, a near CTA size and a
    persistent grid from its sets, and the batch still matches the
    single-geometry FP64 path afterwards."""
    ctx = S.sbio_ctx_create(0, 0)
    specs = [(9, 8), (25, 12), (14, 16)]
    susps = [I.rsa_suspension(M, 0.15, 700 + k, p, name=f"bt{k}") for k, (M, p) in enumerate(specs)]
    geoms = [S.Geometry(ctx, s, precision=S.SBIO_MIXED) for s in susps]
    sig, mu, ref = [], [], []
    for s, g in zip(susps, geoms):
        c = I.config_coefficients(s, 9)
        sig.append(torch.from_numpy(c[0]).cuda())
        mu.append(torch.from_numpy(c[1]).cuda())
        So = torch.empty(g.N, dtype=torch.float64, device="cuda")
        Do = torch.empty_like(So)
        S.sbio_geom_set_precision(g.h, S.SBIO_FP64)
        S.sbio_apply_laplace(g.h, sig[-1], mu[-1], So, Do)
        S.sbio_geom_set_precision(g.h, S.SBIO_MIXED)
        ref.append((So.cpu().numpy(), Do.cpu().numpy()))
    outS = [torch.empty(g.N, dtype=torch.float64, device="cuda") for g in geoms]
    outD = [torch.empty_like(o) for o in outS]
    b = S.sbio_batch_create(ctx, geoms)
    tt, nb, cps, ms = S.sbio_batch_autotune(b, sig, mu, outS, outD)
    assert tt in (1, 2, 4, 8, -2, -4, -8) and nb in (64, 128) and cps in (2, 3, 4, 5, 6, 8) and ms > 0
    assert S.sbio_batch_info(b)["far_tt"] == tt
    for o in outS + outD:
        o.fill_(float("nan"))
    S.sbio_batch_apply(b, sig, mu, outS, outD)
    torch.cuda.synchronize()
    for k, (Sr, Dr) in enumerate(ref):
        assert relerr(outS[k].cpu().numpy(), Sr) < TOLMIX
        assert relerr(outD[k].cpu().numpy(), Dr) < TOLMIX
    S.sbio_batch_destroy(b)
    for g in geoms:
        g.close()
    S.sbio_ctx_destroy(ctx)
