"""GPU forward transform and exterior Dirichlet / Neumann solves (C ABI
sbio_forward_transform, sbio_solve_dirichlet, sbio_solve_neumann) against
the oracle's transform and dense solves, and the paper's point-charge test
run end to end on the GPU (solve, then evaluate at shell points)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import geometry as OG
from oracle import solve as OS
from paper_2506_20809_gb300 import inputs as I

pytestmark = pytest.mark.gpu
COMP = {"CI": 0, "etaCI": 1, "S": 2, "etaS": 3}


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


def charges_setup(p, seed=0):
    rng = np.random.default_rng(seed)
    kind = np.array([0, 1, 0], np.int32)
    A = np.array([0.8, 1.3, 0.75])
    C = np.array([1.4, 0.72, 1.35])
    cen = np.array([[0.0, 0, 0], [5, 0, 0], [3.2, 3.2, 3.2]])
    quat = I.random_quaternions(rng, 3)
    R = I._quat_to_matrix(quat)
    xs = np.concatenate([cen[i] + (rng.uniform(-0.05, 0.05, (2, 3)) * np.array([A[i], A[i], C[i]])) @ R[i].T
                         for i in range(3)])
    qs = rng.uniform(-0.5, 0.5, len(xs))
    return I.Suspension(kind, A, C, cen, quat, p), xs, qs


def f_of(xs, qs, x):
    return (qs / (4 * np.pi * np.linalg.norm(np.atleast_2d(x)[:, None, :] - xs[None], axis=-1))).sum(1)


def dfdn_of(xs, qs, x, n):
    r = x[:, None, :] - xs[None]
    d = np.linalg.norm(r, axis=-1)
    return -(qs * np.einsum("tsk,tk->ts", r, n) / (4 * np.pi * d ** 3)).sum(1)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_forward_transform(S, ctx):
    s = I.rsa_suspension(6, 0.12, 31, 9, ar_range=(1.2, 4.0))
    g = S.Geometry(ctx, s)
    og = OG.SuspensionGeom.from_suspension(s)
    vals = np.random.default_rng(0).standard_normal(g.N)
    B = OS.BVPOracle(og)
    for mod in (False, True):
        out = torch.empty((s.M, 100), dtype=torch.float64, device="cuda")
        S.sbio_forward_transform(g.h, dev(vals), out, mod)
        torch.cuda.synchronize()
        assert rel(out.cpu().numpy(), B.transform(vals, mod)) < 1e-13
    g.close()


@pytest.mark.parametrize("completion", ["CI", "etaCI", "S", "etaS"])
def test_dirichlet_matches_dense_oracle(S, ctx, completion):
    p = 6
    s, xs, qs = charges_setup(p)
    g = S.Geometry(ctx, s)
    og = OG.SuspensionGeom.from_suspension(s)
    nc = (p + 1) ** 2
    mu_r, st_r, q_r = OS.BVPOracle(og).solve_dirichlet(f_of(xs, qs, og.x), completion)
    mu = torch.empty((3, nc), dtype=torch.float64, device="cuda")
    st = torch.empty_like(mu)
    q = torch.empty(3, dtype=torch.float64, device="cuda")
    info = S.sbio_solve_dirichlet(g.h, dev(f_of(xs, qs, og.x)), mu, COMP[completion], tol=1e-13, max_iter=400,
                                  restart=60, sigma_tilde_out=st, charges_out=q)
    assert info["converged"] and info["rel_residual"] < 1e-12
    assert rel(mu.cpu().numpy(), mu_r) < 1e-9
    if completion in ("S", "etaS"):
        assert rel(st.cpu().numpy(), st_r) < 1e-9
        assert np.all(q.cpu().numpy() == 0)
    else:
        assert rel(q.cpu().numpy(), q_r) < 1e-9
        assert np.all(st.cpu().numpy() == 0)
    g.close()


def test_neumann_matches_dense_oracle(S, ctx):
    p = 6
    s, xs, qs = charges_setup(p, seed=3)
    g = S.Geometry(ctx, s)
    og = OG.SuspensionGeom.from_suspension(s)
    rho_r = OS.BVPOracle(og).solve_neumann(dfdn_of(xs, qs, og.x, og.nrm))
    rho = torch.empty((3, (p + 1) ** 2), dtype=torch.float64, device="cuda")
    info = S.sbio_solve_neumann(g.h, dev(dfdn_of(xs, qs, og.x, og.nrm)), rho, tol=1e-13, max_iter=400, restart=60)
    assert info["converged"]
    assert rel(rho.cpu().numpy(), rho_r) < 1e-9
    g.close()


def test_point_charge_problem_end_to_end(S, ctx):
    """The paper's test on the GPU: solve, then evaluate u at shells
    1e-1 .. 1e-6 outside the surfaces; spectral decay of the error in p for
    the Dirichlet (etaS) and Neumann solves, and restarts do not change the
    answer."""
    errs = {"D": [], "N": []}
    for p in (6, 10, 14):
        s, xs, qs = charges_setup(p, seed=5)
        g = S.Geometry(ctx, s)
        xyz, nrm, _ = S.sbio_geom_nodes(g.h)
        X = I.shell_points(s, per_particle=6, seed=2)
        ts = S.TargetSet(g, X)
        ref = f_of(xs, qs, X)
        nc = (p + 1) ** 2
        mu = torch.empty((3, nc), dtype=torch.float64, device="cuda")
        st = torch.empty_like(mu)
        q = torch.empty(3, dtype=torch.float64, device="cuda")
        info = S.sbio_solve_dirichlet(g.h, dev(f_of(xs, qs, xyz)), mu, COMP["etaS"], tol=1e-12, sigma_tilde_out=st,
                                      charges_out=q)
        assert info["converged"]
        Su = torch.empty(ts.T, dtype=torch.float64, device="cuda")
        Du = torch.empty_like(Su)
        S.sbio_eval_targets(ts.h, st, mu, Su, Du)
        torch.cuda.synchronize()
        errs["D"].append(rel((Su + Du).cpu().numpy(), ref))
        rho = torch.empty_like(mu)
        info = S.sbio_solve_neumann(g.h, dev(dfdn_of(xs, qs, xyz, nrm)), rho, tol=1e-12)
        assert info["converged"]
        S.sbio_eval_targets(ts.h, rho, None, Su, None)
        torch.cuda.synchronize()
        errs["N"].append(rel(Su.cpu().numpy(), ref))
        if p == 10:
            mu2 = torch.empty_like(mu)
            info2 = S.sbio_solve_dirichlet(g.h, dev(f_of(xs, qs, xyz)), mu2, COMP["etaS"], tol=1e-12, restart=5)
            assert info2["converged"] and info2["restarts"] > 0
            assert rel(mu2.cpu().numpy(), mu.cpu().numpy()) < 1e-9
        ts.close()
        g.close()
    for k, e in errs.items():
        assert e[2] < 1e-4 and e[2] < e[1] < e[0], (k, e)


def test_mixed_precision_solve(S, ctx):
    s, xs, qs = charges_setup(10, seed=7)
    g = S.Geometry(ctx, s)
    xyz, _, _ = S.sbio_geom_nodes(g.h)
    out = []
    # the mixed operator carries FP32 rounding (~1e-7 relative), which bounds
    # the residual GMRES can reach with it
    for prec, tol in ((S.SBIO_FP64, 1e-10), (S.SBIO_MIXED, 1e-6)):
        S.sbio_geom_set_precision(g.h, prec)
        mu = torch.empty((3, 121), dtype=torch.float64, device="cuda")
        info = S.sbio_solve_dirichlet(g.h, dev(f_of(xs, qs, xyz)), mu, COMP["etaS"], tol=tol)
        print(prec, info)
        assert info["converged"]
        out.append(mu.cpu().numpy())
    assert rel(out[1], out[0]) < 1e-5
    g.close()


def test_invalid_arguments(S, ctx):
    s, xs, qs = charges_setup(4)
    g = S.Geometry(ctx, s)
    f = torch.zeros(g.N, dtype=torch.float64, device="cuda")
    mu = torch.zeros((3, 25), dtype=torch.float64, device="cuda")
    for kw in ({"completion": 9}, {"tol": 0.0}, {"restart": 0}):
        with pytest.raises(S.SbioError) as e:
            S.sbio_solve_dirichlet(g.h, f, mu, **kw)
        assert e.value.code == S.SBIO_EINVAL
    # zero data: zero solution, converged at once
    info = S.sbio_solve_dirichlet(g.h, f, mu)
    assert info["converged"] and info["iterations"] == 0 and float(mu.abs().max()) == 0.0
    g.close()
