"""GPU parity of the Laplace apply (C ABI) against the CPU oracle.

FP64 path: normwise relative error <= 1e-10 against the oracle's O-method
(same nodes, same near sets, analytic self + near, smooth far quadrature).
Mixed path: normwise relative error <= 1e-6 against the GPU FP64 path."""
import math

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
    c = S.sbio_ctx_create(0, 0)
    yield c


def gpu_apply(S, geom, sig, mu, parts=7, precision=None):
    if precision is not None:
        S.sbio_geom_set_precision(geom.h, precision)
    sg = None if sig is None else torch.from_numpy(np.ascontiguousarray(sig)).cuda()
    mg = None if mu is None else torch.from_numpy(np.ascontiguousarray(mu)).cuda()
    So = None if sig is None else torch.full((geom.N,), float("nan"), dtype=torch.float64, device="cuda")
    Do = None if mu is None else torch.full((geom.N,), float("nan"), dtype=torch.float64, device="cuda")
    S.sbio_apply_laplace_parts(geom.h, sg, mg, So, Do, parts)
    torch.cuda.synchronize()
    return (None if So is None else So.cpu().numpy(), None if Do is None else Do.cpu().numpy())


def small_suspension(seed, M=3, p=5, ar=(1.3, 4.0)):
    s = I.rsa_suspension(M, 0.12, seed, p, ar_range=ar, min_gap=0.05, name="small")
    return s


@pytest.fixture(scope="module")
def lattice(S, ctx):
    s = I.config_suspension(1)
    c = I.config_coefficients(s, 0)
    g = S.Geometry(ctx, s)
    og = OG.SuspensionGeom.from_suspension(s)
    return s, c, g, og, OL.LaplaceOracle(og)


def test_nodes_and_near_sets_match_oracle(S, lattice):
    s, c, g, og, O = lattice
    xyz, nrm, w = S.sbio_geom_nodes(g.h)
    np.testing.assert_allclose(xyz, og.x, atol=1e-13)
    np.testing.assert_allclose(nrm, np.concatenate([P.nrm for P in og.parts]), atol=1e-13)
    np.testing.assert_allclose(w, np.concatenate([P.w for P in og.parts]), rtol=1e-13)
    t, src = S.sbio_geom_near_pairs(g.h)
    lib_pairs = set(zip(t.tolist(), src.tolist()))
    nt, ns = np.nonzero(og.near_matrix())
    assert lib_pairs == set(zip(nt.tolist(), ns.tolist()))
    assert g.n_far == O.far_pair_count()


@pytest.mark.parametrize("parts,name", [(1, "self"), (2, "near"), (4, "far"), (7, "all")])
def test_lattice_fp64_parts(S, lattice, parts, name):
    s, c, g, og, O = lattice
    sel = {1: ("self",), 2: ("near",), 4: ("far",), 7: ("self", "near", "far")}[parts]
    Sr, Dr = O.apply(c[0], c[1], "method", parts=sel)
    Sg, Dg = gpu_apply(S, g, c[0], c[1], parts, S.SBIO_FP64)
    assert OL.normwise_rel_err(Sg, Sr) < TOL64, name
    assert OL.normwise_rel_err(Dg, Dr) < TOL64, name


def test_lattice_mixed(S, lattice):
    s, c, g, og, O = lattice
    S64, D64 = gpu_apply(S, g, c[0], c[1], 7, S.SBIO_FP64)
    Sm, Dm = gpu_apply(S, g, c[0], c[1], 7, S.SBIO_MIXED)
    S.sbio_geom_set_precision(g.h, S.SBIO_FP64)
    assert OL.normwise_rel_err(Sm, S64) < TOLMIX
    assert OL.normwise_rel_err(Dm, D64) < TOLMIX


@pytest.mark.parametrize("tt,splits", [(1, 1), (2, 3), (4, 0), (1, 7), (8, 0), (8, 5), (-2, 0), (-4, 3), (-8, 0)])
def test_launch_shapes_agree(S, lattice, tt, splits):
    """Far-field launch shapes (targets per thread, source splits) change only
    the summation order."""
    s, c, g, og, O = lattice
    S64, D64 = gpu_apply(S, g, c[0], c[1], 7, S.SBIO_FP64)
    S.sbio_geom_set_launch_shape(g.h, tt, splits)
    S64b, D64b = gpu_apply(S, g, c[0], c[1], 7, S.SBIO_FP64)
    Sm, Dm = gpu_apply(S, g, c[0], c[1], 7, S.SBIO_MIXED)
    S.sbio_geom_set_launch_shape(g.h, 2, 0)
    S.sbio_geom_set_precision(g.h, S.SBIO_FP64)
    assert OL.normwise_rel_err(S64b, S64) < 1e-13 and OL.normwise_rel_err(D64b, D64) < 1e-13
    assert OL.normwise_rel_err(Sm, S64) < TOLMIX and OL.normwise_rel_err(Dm, D64) < TOLMIX


def test_overlap_matches_in_order(S, poly200):
    """Near kernels on the forked high-priority stream give the in-order result."""
    s, c, g, og = poly200
    S.sbio_geom_set_precision(g.h, S.SBIO_MIXED)
    S.sbio_geom_set_overlap(g.h, True)
    So, Do = gpu_apply(S, g, c[0], c[1], 7)
    S.sbio_geom_set_overlap(g.h, False)
    Si, Di = gpu_apply(S, g, c[0], c[1], 7)
    S.sbio_geom_set_overlap(g.h, True)
    S.sbio_geom_set_precision(g.h, S.SBIO_FP64)
    assert OL.normwise_rel_err(So, Si) < 1e-12 and OL.normwise_rel_err(Do, Di) < 1e-12


def test_autotune_keeps_results(S, lattice):
    s, c, g, og, O = lattice
    S.sbio_geom_set_precision(g.h, S.SBIO_MIXED)
    try:
        tt, sp, ms = S.sbio_geom_autotune(g.h)
        assert tt in (1, 2, 4, 8, -2, -4, -8) and sp >= 1 and ms > 0
        Sm, Dm = gpu_apply(S, g, c[0], c[1], 7, S.SBIO_MIXED)
        S64, D64 = gpu_apply(S, g, c[0], c[1], 7, S.SBIO_FP64)
        assert OL.normwise_rel_err(Sm, S64) < TOLMIX and OL.normwise_rel_err(Dm, D64) < TOLMIX
    finally:
        S.sbio_geom_set_launch_shape(g.h, 2, 0)
        S.sbio_geom_set_precision(g.h, S.SBIO_FP64)


def test_single_operators(S, lattice):
    s, c, g, og, O = lattice
    Sr, _ = O.apply(c[0], None, "method")
    _, Dr = O.apply(None, c[1], "method")
    Sg, _ = gpu_apply(S, g, c[0], None, 7, S.SBIO_FP64)
    _, Dg = gpu_apply(S, g, None, c[1], 7, S.SBIO_FP64)
    assert OL.normwise_rel_err(Sg, Sr) < TOL64
    assert OL.normwise_rel_err(Dg, Dr) < TOL64


def test_host_memory_entry_point(S, lattice):
    s, c, g, og, O = lattice
    Sd, Dd = gpu_apply(S, g, c[0], c[1], 7, S.SBIO_FP64)
    Sh = np.zeros(g.N)
    Dh = np.zeros(g.N)
    S.sbio_apply_laplace_host(g.h, np.ascontiguousarray(c[0]), np.ascontiguousarray(c[1]), Sh, Dh)
    np.testing.assert_allclose(Sh, Sd, rtol=0, atol=1e-14 * np.abs(Sd).max())
    np.testing.assert_allclose(Dh, Dd, rtol=0, atol=1e-14 * np.abs(Dd).max())


@pytest.mark.parametrize("p", [1, 2, 3, 5, 7, 10, 13, 16, 19, 22, 24])
def test_orders_ragged(S, ctx, p):
    """Every compiled order, on a close 3-particle cluster (ragged tiles)."""
    s = small_suspension(100 + p, M=3, p=p)
    rng = np.random.default_rng(p)
    sig = I.coefficients(rng, 3, p)
    mu = I.coefficients(rng, 3, p)
    g = S.Geometry(ctx, s, near_factor=2.0)
    O = OL.LaplaceOracle(OG.SuspensionGeom.from_suspension(s, near_factor=2.0))
    Sr, Dr = O.apply(sig, mu, "method")
    Sg, Dg = gpu_apply(S, g, sig, mu, 7, S.SBIO_FP64)
    assert g.n_near > 0
    assert OL.normwise_rel_err(Sg, Sr) < TOL64
    assert OL.normwise_rel_err(Dg, Dr) < TOL64
    g.close()


def test_single_particle_self_only(S, ctx):
    s = I.Suspension(np.array([1], np.int32), np.array([1.3]), np.array([0.5]), np.zeros((1, 3)),
                     np.array([[0.9, 0.1, -0.3, 0.2]]) / np.linalg.norm([0.9, 0.1, -0.3, 0.2]), 6)
    rng = np.random.default_rng(0)
    sig = I.coefficients(rng, 1, 6)
    mu = I.coefficients(rng, 1, 6)
    g = S.Geometry(ctx, s)
    O = OL.LaplaceOracle(OG.SuspensionGeom.from_suspension(s))
    Sr, Dr = O.apply(sig, mu, "method")
    Sg, Dg = gpu_apply(S, g, sig, mu)
    assert g.n_near == 0 and g.n_far == 0
    assert OL.normwise_rel_err(Sg, Sr) < TOL64 and OL.normwise_rel_err(Dg, Dr) < TOL64
    # Gauss: D[1] = -1/2 on the surface
    mu1 = np.zeros_like(mu)
    mu1[0, 0] = math.sqrt(4 * math.pi)
    _, D1 = gpu_apply(S, g, None, mu1)
    np.testing.assert_allclose(D1, -0.5, atol=1e-13)
    g.close()


def test_paper_style_nonuniform_phi_grid(S, ctx):
    """n_phi = 2p as printed in Sec. 4 (aliasing of sin(p phi) is the user's)."""
    s = small_suspension(7, M=3, p=6)
    rng = np.random.default_rng(1)
    sig = I.coefficients(rng, 3, 6)
    mu = I.coefficients(rng, 3, 6)
    g = S.Geometry(ctx, s, n_phi=12)
    O = OL.LaplaceOracle(OG.SuspensionGeom.from_suspension(s, n_phi=12))
    Sr, Dr = O.apply(sig, mu, "method")
    Sg, Dg = gpu_apply(S, g, sig, mu)
    assert OL.normwise_rel_err(Sg, Sr) < TOL64 and OL.normwise_rel_err(Dg, Dr) < TOL64
    g.close()


def test_invalid_inputs(S, ctx):
    base = small_suspension(3, M=2, p=4)
    sph = S.make_spheroids(base.kind, base.A, base.C, base.center, base.quat)
    with pytest.raises(S.SbioError) as e:
        S.sbio_geom_create(ctx, sph, 0)
    assert e.value.code == S.SBIO_EINVAL
    with pytest.raises(S.SbioError) as e:
        S.sbio_geom_create(ctx, sph, 4, far_upsample=2)
    assert e.value.code == S.SBIO_ENOTSUP
    bad = S.make_spheroids(base.kind, base.A, base.C, np.zeros((2, 3)), base.quat)   # same centre
    with pytest.raises(S.SbioError) as e:
        S.sbio_geom_create(ctx, bad, 4)
    assert e.value.code == S.SBIO_EOVERLAP
    sphere = S.make_spheroids([0], [1.0], [1.0], [[0, 0, 0]], [[1, 0, 0, 0]])
    with pytest.raises(S.SbioError) as e:
        S.sbio_geom_create(ctx, sphere, 4)
    assert e.value.code == S.SBIO_EINVAL
    small_budget = S.sbio_ctx_create(0, 4096)
    with pytest.raises(S.SbioError) as e:
        S.sbio_geom_create(small_budget, sph, 4)
    assert e.value.code == S.SBIO_ENOMEM
    assert S.sbio_ctx_mem_used(small_budget) == 0
    S.sbio_ctx_destroy(small_budget)


@pytest.fixture(scope="module")
def poly200(S, ctx):
    s = I.config_suspension(2)
    c = I.config_coefficients(s, 0)
    g = S.Geometry(ctx, s)
    og = OG.SuspensionGeom.from_suspension(s)
    return s, c, g, og


def test_poly200_sampled_fp64(S, poly200):
    """Full 200-spheroid, p = 16 workload in the benchmark's launch
    configuration; the oracle evaluates a sample of targets one by one."""
    s, c, g, og = poly200
    Sg, Dg = gpu_apply(S, g, c[0], c[1], 7, S.SBIO_FP64)
    rng = np.random.default_rng(0)
    tg = np.sort(rng.choice(g.N, 240, replace=False))
    O = OL.LaplaceOracle(og)
    Sr, Dr = O.apply(c[0], c[1], "method", targets=tg)
    # normwise over the sample, relative to the max over all targets
    assert np.max(np.abs(Sg[tg] - Sr)) / np.max(np.abs(Sg)) < TOL64
    assert np.max(np.abs(Dg[tg] - Dr)) / np.max(np.abs(Dg)) < TOL64


def test_poly200_mixed_vs_fp64(S, poly200):
    s, c, g, og = poly200
    S64, D64 = gpu_apply(S, g, c[0], c[1], 7, S.SBIO_FP64)
    Sm, Dm = gpu_apply(S, g, c[0], c[1], 7, S.SBIO_MIXED)
    S.sbio_geom_set_precision(g.h, S.SBIO_FP64)
    eS, eD = OL.normwise_rel_err(Sm, S64), OL.normwise_rel_err(Dm, D64)
    print(f"mixed vs fp64: S {eS:.3e} D {eD:.3e}")
    assert eS < TOLMIX and eD < TOLMIX


def gpu_limit(S, geom, sig, mu, side, deriv=False):
    sg = None if sig is None else torch.from_numpy(np.ascontiguousarray(sig)).cuda()
    mg = None if mu is None else torch.from_numpy(np.ascontiguousarray(mu)).cuda()
    So = None if sig is None else torch.full((geom.N,), float("nan"), dtype=torch.float64, device="cuda")
    Do = None if mu is None else torch.full((geom.N,), float("nan"), dtype=torch.float64, device="cuda")
    fn = S.sbio_apply_laplace_deriv_limit if deriv else S.sbio_apply_laplace_limit
    fn(geom.h, sg, mg, So, Do, side)
    torch.cuda.synchronize()
    return (None if So is None else So.cpu().numpy(), None if Do is None else Do.cpu().numpy())


def test_one_sided_limits(S, lattice):
    """D+- = D +- mu/2 and S'+- = S' -+ sigma/2 at every node (the density
    values from the oracle's synthesis); S and D' are the same on both sides."""
    s, c, g, og, O = lattice
    S.sbio_geom_set_precision(g.h, S.SBIO_FP64)
    sval = np.concatenate([OL.density_values(P, c[0][i], None)[0] for i, P in enumerate(og.parts)])
    mval = np.concatenate([OL.density_values(P, None, c[1][i])[1] for i, P in enumerate(og.parts)])
    S0, D0 = gpu_limit(S, g, c[0], c[1], 0)
    Sp0, Dp0 = gpu_limit(S, g, c[0], c[1], 0, deriv=True)
    for side in (1, -1):
        Ss, Ds = gpu_limit(S, g, c[0], c[1], side)
        assert np.max(np.abs(Ss - S0)) <= 1e-13 * np.max(np.abs(S0))
        assert np.max(np.abs(Ds - (D0 + 0.5 * side * mval))) <= 1e-13 * np.max(np.abs(D0))
        Sps, Dps = gpu_limit(S, g, c[0], c[1], side, deriv=True)
        assert np.max(np.abs(Sps - (Sp0 - 0.5 * side * sval))) <= 1e-12 * np.max(np.abs(Sp0))
        assert np.max(np.abs(Dps - Dp0)) <= 1e-13 * np.max(np.abs(Dp0))
    with pytest.raises(S.SbioError) as e:
        gpu_limit(S, g, c[0], c[1], 2)
    assert e.value.code == S.SBIO_EINVAL


@pytest.mark.parametrize("kind,A,C", [(0, 0.7, 1.6), (1, 1.5, 0.6)])
def test_limits_gauss_and_conductor(S, ctx, kind, A, C):
    """One spheroid of each kind.  Gauss's law for mu = 1: D+ = 0 and D- = -1
    at every node; the conductor (equilibrium) density: S'+ = -sigma and
    S'- = 0."""
    q = np.array([0.8, 0.1, -0.5, 0.3])
    one = I.Suspension(np.array([kind], np.int32), np.array([A]), np.array([C]), np.zeros((1, 3)),
                       (q / np.linalg.norm(q))[None], 8)
    mu = np.zeros((1, 81))
    mu[0, 0] = math.sqrt(4 * math.pi)   # mu = 1 (Y_00 = 1 / sqrt(4 pi))
    sig = np.zeros((1, 81))
    sig[0, 0] = 1.0
    g = S.Geometry(ctx, one, precision=S.SBIO_FP64)
    _, Dp = gpu_limit(S, g, None, mu, 1)
    _, Dm = gpu_limit(S, g, None, mu, -1)
    assert np.max(np.abs(Dp)) < 1e-12
    assert np.max(np.abs(Dm + 1.0)) < 1e-12
    og = OG.SuspensionGeom.from_suspension(one)
    sval, _ = OL.density_values(og.parts[0], sig[0], None)
    Spp, _ = gpu_limit(S, g, sig, None, 1, deriv=True)
    Spm, _ = gpu_limit(S, g, sig, None, -1, deriv=True)
    assert np.max(np.abs(Spp + sval)) < 1e-12 * np.max(np.abs(sval))
    assert np.max(np.abs(Spm)) < 1e-12 * np.max(np.abs(sval))
    g.close()
