"""The treecode far field (C ABI sbio_geom_set_far_method with
SBIO_FAR_TREE) against the direct far sum it replaces: every far (target,
source node) pair covered exactly once, the whole mixed apply within the
stated bound of the plain FP64 GPU apply and of the CPU oracle's method on
sampled targets, at the orders and opening angles offered."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import geometry as OG
from oracle import laplace as OL
from paper_2506_20809_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOLMIX = 1e-6
# stated bounds of the treecode apply against FP64 (normwise), per (order, theta)
TREE_BOUND = {(16, 0.5): 1e-6, (12, 0.5): 3e-6, (8, 0.4): 3e-5}


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


def _apply(S, g, c):
    sig = torch.from_numpy(c[0]).cuda()
    mu = torch.from_numpy(c[1]).cuda()
    So = torch.full((g.N,), float("nan"), dtype=torch.float64, device="cuda")
    Do = torch.full_like(So, float("nan"))
    S.sbio_apply_laplace(g.h, sig, mu, So, Do)
    torch.cuda.synchronize()
    return So.cpu().numpy(), Do.cpu().numpy()


@pytest.mark.parametrize("M,p,seed", [(60, 8, 31), (120, 12, 32), (90, 16, 33), (50, 20, 34)])
def test_tree_matches_fp64_direct(S, ctx, M, p, seed):
    s = I.rsa_suspension(M, 0.20, seed, p, name="tree")
    c = I.config_coefficients(s, seed)
    g = S.Geometry(ctx, s, precision=S.SBIO_FP64)
    S64, D64 = _apply(S, g, c)
    S.sbio_geom_set_precision(g.h, S.SBIO_MIXED)
    for (order, theta), bound in TREE_BOUND.items():
        S.sbio_geom_set_far_method(g.h, S.SBIO_FAR_TREE, theta, order)
        info = S.sbio_geom_tree_info(g.h)
        assert info["nodes"] == 2 * M - 1
        assert info["m2p_source_pairs"] + info["direct_pairs"] == g.n_far
        # evaluations split by order, none above the treecode's order
        oc = S.sbio_geom_tree_order_counts(g.h, S.SBIO_OP_LAPLACE)
        ocs = S.sbio_geom_tree_order_counts(g.h, S.SBIO_OP_STOKES)
        assert sum(oc.values()) == info["m2p_pairs"] == sum(ocs.values())
        assert all(v == 0 for e, v in oc.items() if e > order)
        assert all(v == 0 for e, v in ocs.items() if e > order)
        # the Stokes lists keep a tenfold margin: never a lower order than Laplace's
        assert ocs[8] <= oc[8] and ocs[8] + ocs[12] <= oc[8] + oc[12]
        if order == 16 and M >= 90:
            assert oc[8] > 0 and oc[12] > 0 and oc[16] > 0
        with pytest.raises(S.SbioError):
            S.sbio_geom_tree_order_counts(g.h, 7)
        St, Dt = _apply(S, g, c)
        eS, eD = OL.normwise_rel_err(St, S64), OL.normwise_rel_err(Dt, D64)
        print(f"M={M} p={p} order={order} theta={theta}: S {eS:.2e} D {eD:.2e}, "
              f"m2p {info['m2p_pairs']:.3e} direct {info['direct_pairs']:.3e}")
        assert eS < bound and eD < bound, (order, theta, eS, eD)
    S.sbio_geom_set_far_method(g.h, S.SBIO_FAR_DIRECT)
    Sd, Dd = _apply(S, g, c)
    assert OL.normwise_rel_err(Sd, S64) < TOLMIX and OL.normwise_rel_err(Dd, D64) < TOLMIX
    g.close()


def test_tree_against_oracle_sampled(S, ctx):
    """A 400-particle suspension of the 200-particle recipe (p = 12): the
    treecode apply against the oracle's method on sampled targets."""
    s = I.rsa_suspension(400, 0.20, 41, 12, name="tree400")
    c = I.config_coefficients(s, 2)
    g = S.Geometry(ctx, s, precision=S.SBIO_MIXED)
    S.sbio_geom_set_far_method(g.h, S.SBIO_FAR_TREE, 0.5, 16)
    St, Dt = _apply(S, g, c)
    og = OG.SuspensionGeom.from_suspension(s)
    tg = np.sort(np.random.default_rng(5).choice(g.N, 40, replace=False))
    Sr, Dr = OL.LaplaceOracle(og).apply(c[0], c[1], "method", targets=tg)
    eS = np.max(np.abs(St[tg] - Sr)) / np.max(np.abs(Sr))
    eD = np.max(np.abs(Dt[tg] - Dr)) / np.max(np.abs(Dr))
    print(f"tree400 vs oracle: S {eS:.2e} D {eD:.2e}")
    assert eS < TREE_BOUND[(16, 0.5)] and eD < TREE_BOUND[(16, 0.5)]
    g.close()


def test_tree_single_operator_and_fp64_keep_direct(S, ctx):
    """S-only applies and FP64 geometries use the direct sum: identical to the
    direct results."""
    s = I.rsa_suspension(30, 0.2, 43, 8, name="tree30")
    c = I.config_coefficients(s, 1)
    g = S.Geometry(ctx, s, precision=S.SBIO_FP64)
    S64, D64 = _apply(S, g, c)
    S.sbio_geom_set_far_method(g.h, S.SBIO_FAR_TREE, 0.5, 16)
    S64t, D64t = _apply(S, g, c)
    assert np.array_equal(np.isnan(S64t), np.isnan(S64))
    assert OL.normwise_rel_err(S64t, S64) < 1e-13 and OL.normwise_rel_err(D64t, D64) < 1e-13
    with pytest.raises(S.SbioError) as e:
        S.sbio_geom_set_far_method(g.h, S.SBIO_FAR_TREE, 1.5, 16)
    assert e.value.code == S.SBIO_EINVAL
    with pytest.raises(S.SbioError):
        S.sbio_geom_set_far_method(g.h, S.SBIO_FAR_TREE, 0.5, 10)
    g.close()


def test_batch_with_treecode_suspensions(S, ctx):
    """A batch mixing treecode and direct far fields (one CUDA graph) gives
    each suspension's FP64 result within the treecode bound."""
    specs = [(40, 8), (120, 12), (15, 16)]
    susps = [I.rsa_suspension(M, 0.2, 800 + k, p, name=f"tb{k}") for k, (M, p) in enumerate(specs)]
    geoms = [S.Geometry(ctx, s, precision=S.SBIO_MIXED) for s in susps]
    sig, mu, ref = [], [], []
    for s, g in zip(susps, geoms):
        c = I.config_coefficients(s, 4)
        sig.append(torch.from_numpy(c[0]).cuda())
        mu.append(torch.from_numpy(c[1]).cuda())
        S.sbio_geom_set_precision(g.h, S.SBIO_FP64)
        ref.append(_apply(S, g, c))
        S.sbio_geom_set_precision(g.h, S.SBIO_MIXED)
    S.sbio_geom_set_far_method(geoms[0].h, S.SBIO_FAR_TREE, 0.5, 16)
    S.sbio_geom_set_far_method(geoms[1].h, S.SBIO_FAR_TREE, 0.5, 16)
    outS = [torch.full((g.N,), float("nan"), dtype=torch.float64, device="cuda") for g in geoms]
    outD = [torch.full_like(o, float("nan")) for o in outS]
    b = S.sbio_batch_create(ctx, geoms)
    for _ in range(2):                                  # capture, then replay
        S.sbio_batch_apply(b, sig, mu, outS, outD)
        torch.cuda.synchronize()
        for k, (Sr, Dr) in enumerate(ref):
            assert OL.normwise_rel_err(outS[k].cpu().numpy(), Sr) < TREE_BOUND[(16, 0.5)]
            assert OL.normwise_rel_err(outD[k].cpu().numpy(), Dr) < TREE_BOUND[(16, 0.5)]
    S.sbio_batch_destroy(b)
    for g in geoms:
        g.close()


@pytest.mark.parametrize("M", [1, 2, 5])
def test_tree_tiny_suspensions(S, ctx, M):
    """One, two and five particles: the tree degenerates (a lone leaf, a
    root over two leaves) and the far field must still match the direct sum
    (with one particle there is none)."""
    s = I.rsa_suspension(M, 0.1, 900 + M, 6, name="tiny")
    c = I.config_coefficients(s, M)
    g = S.Geometry(ctx, s, precision=S.SBIO_FP64)
    S64, D64 = _apply(S, g, c)
    S.sbio_geom_set_precision(g.h, S.SBIO_MIXED)
    S.sbio_geom_set_far_method(g.h, S.SBIO_FAR_TREE, 0.5, 16)
    info = S.sbio_geom_tree_info(g.h)
    assert info["nodes"] == 2 * M - 1
    assert info["m2p_source_pairs"] + info["direct_pairs"] == g.n_far
    St, Dt = _apply(S, g, c)
    assert OL.normwise_rel_err(St, S64) < TREE_BOUND[(16, 0.5)]
    assert OL.normwise_rel_err(Dt, D64) < TREE_BOUND[(16, 0.5)]
    g.close()


def test_tree_settings_switch_and_rebuild(S, ctx):
    """Changing order and opening angle rebuilds the lists, returning to the
    direct sum restores its result exactly, and timing the phases works."""
    s = I.rsa_suspension(80, 0.2, 910, 8, name="switch")
    c = I.config_coefficients(s, 2)
    g = S.Geometry(ctx, s, precision=S.SBIO_MIXED)
    Sd, Dd = _apply(S, g, c)
    S.sbio_geom_set_far_method(g.h, S.SBIO_FAR_TREE, 0.5, 16)
    a = S.sbio_geom_tree_info(g.h)
    S.sbio_geom_set_far_method(g.h, S.SBIO_FAR_TREE, 0.3, 12)
    b = S.sbio_geom_tree_info(g.h)
    assert b["direct_pairs"] > a["direct_pairs"]          # a smaller angle opens more nodes
    assert b["m2p_source_pairs"] + b["direct_pairs"] == g.n_far
    S.sbio_geom_enable_timing(g.h, True)
    St, Dt = _apply(S, g, c)
    ph = S.sbio_geom_tree_phase_times(g.h)
    S.sbio_geom_enable_timing(g.h, False)
    assert all(x >= 0 for x in ph) and sum(ph) > 0
    assert OL.normwise_rel_err(St, Sd) < TREE_BOUND[(12, 0.5)]
    S.sbio_geom_set_far_method(g.h, S.SBIO_FAR_DIRECT)
    Sd2, Dd2 = _apply(S, g, c)
    assert np.array_equal(Sd2, Sd) or OL.normwise_rel_err(Sd2, Sd) < 1e-13
    with pytest.raises(S.SbioError):
        S.sbio_geom_tree_info(g.h)
    g.close()


def _stokes(S, g, f):
    u = torch.full((g.N, 3), float("nan"), dtype=torch.float64, device="cuda")
    S.sbio_apply_stokes_sl(g.h, torch.from_numpy(np.ascontiguousarray(f)).cuda(), u)
    torch.cuda.synchronize()
    return u.cpu().numpy()


@pytest.mark.parametrize("M,p,seed", [(50, 8, 51), (100, 12, 52), (60, 20, 53)])
def test_stokes_tree_matches_fp64_direct(S, ctx, M, p, seed):
    """The Stokes single layer with the treecode far field (four charge and
    four dipole channels per node) against the plain FP64 direct apply."""
    s = I.rsa_suspension(M, 0.15, seed, p, ar_range=(1.5, 4.0), name="stree")
    f = I.config_coefficients(s, seed, ndens=3).transpose(1, 0, 2).copy()
    g = S.Geometry(ctx, s, precision=S.SBIO_FP64)
    U64 = _stokes(S, g, f)
    S.sbio_geom_set_precision(g.h, S.SBIO_MIXED)
    Ud = _stokes(S, g, f)
    S.sbio_geom_set_far_method(g.h, S.SBIO_FAR_TREE, 0.5, 16)
    Ut = _stokes(S, g, f)
    e = OL.normwise_rel_err(Ut, U64)
    print(f"stokes tree M={M} p={p}: {e:.2e} (direct mixed {OL.normwise_rel_err(Ud, U64):.2e})")
    assert e < TREE_BOUND[(16, 0.5)]
    g.close()


def test_stokes_tree_against_oracle_sampled(S, ctx):
    from oracle import stokes as OSt

    s = I.rsa_suspension(200, 0.15, 61, 10, ar_range=(1.5, 4.0), name="stree200")
    f = I.config_coefficients(s, 3, ndens=3).transpose(1, 0, 2).copy()
    g = S.Geometry(ctx, s, precision=S.SBIO_MIXED)
    S.sbio_geom_set_far_method(g.h, S.SBIO_FAR_TREE, 0.5, 16)
    Ut = _stokes(S, g, f)
    og = OG.SuspensionGeom.from_suspension(s)
    tg = np.sort(np.random.default_rng(8).choice(g.N, 30, replace=False))
    Ur = OSt.StokesOracle(og).apply(f, "method", targets=tg)
    e = np.max(np.abs(Ut[tg] - Ur)) / np.max(np.abs(Ur))
    print(f"stokes tree200 vs oracle: {e:.2e}")
    assert e < TREE_BOUND[(16, 0.5)]
    g.close()


def test_tree_forked_phases_equal_in_order(S, ctx):
    """With overlap on, the treecode's direct part runs on its own stream
    beside the multipole phases and the near kernels beside both; the result
    is the in-order apply's up to the order of the atomic additions.  The
    treecode's near cap is tuned when the treecode is attached, kept apart
    from the direct sum's, and settable."""
    s = I.rsa_suspension(150, 0.20, 71, 12, name="treefork")
    c = I.config_coefficients(s, 71)
    f = I.config_coefficients(s, 72, ndens=3).transpose(1, 0, 2).copy()
    g = S.Geometry(ctx, s, precision=S.SBIO_MIXED)
    S.sbio_geom_set_near_cap(g.h, 1)
    S.sbio_geom_set_far_method(g.h, S.SBIO_FAR_TREE, 0.5, 16)
    assert S.sbio_geom_get_tree_near_cap(g.h) in (0, 1, 2, 3, 4, 8)
    assert S.sbio_geom_get_tuning(g.h)["near_ctas_per_sm"] == 1
    outs = {}
    for cap in (1, 3):
        S.sbio_geom_set_tree_near_cap(g.h, cap)
        assert S.sbio_geom_get_tree_near_cap(g.h) == cap
        S.sbio_geom_set_overlap(g.h, True)
        outs[cap] = _apply(S, g, c) + (_stokes(S, g, f),)
    S.sbio_geom_set_overlap(g.h, False)
    Si, Di = _apply(S, g, c)
    Ui = _stokes(S, g, f)
    for cap, (Sf, Df, Uf) in outs.items():
        assert np.isfinite(Sf).all() and np.isfinite(Df).all() and np.isfinite(Uf).all()
        assert OL.normwise_rel_err(Sf, Si) < 1e-12, cap
        assert OL.normwise_rel_err(Df, Di) < 1e-12, cap
        assert OL.normwise_rel_err(Uf, Ui) < 1e-12, cap
    with pytest.raises(S.SbioError):
        S.sbio_geom_set_tree_near_cap(g.h, -1)
    g.close()
