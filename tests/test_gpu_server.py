"""Serving engine: continuous batching of Laplace and Stokes requests.

Each request's results are the same alone and in a mix of concurrent
requests, and equal to direct applies on a resident geometry; a tight memory
budget still completes every request (admission waits for memory)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2506_20809_gb300 import inputs as I

pytestmark = pytest.mark.gpu
NAPPLY = 3


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as G

    G.build()
    import paper_2506_20809_gb300.sbio as S

    return S


def make_requests():
    reqs = []
    for k, (M, p, op) in enumerate([(6, 6, "laplace"), (9, 8, "stokes"), (14, 8, "laplace"), (5, 12, "stokes"),
                                    (11, 5, "laplace")]):
        s = I.rsa_suspension(M, 0.12, 500 + k, p, name=f"r{k}")
        nc = (p + 1) ** 2
        rng = np.random.default_rng(k)
        nd = 2 if op == "laplace" else 3
        coef = np.stack([I.coefficients(rng, M, p, nd) for _ in range(NAPPLY)])     # (A, M, nd, nc)
        if op == "laplace":
            coef = np.ascontiguousarray(np.transpose(coef, (0, 2, 1, 3)))          # (A, 2, M, nc)
        N = M * (p + 1) * 2 * (p + 1)
        reqs.append({"s": s, "p": p, "op": op, "coef": coef, "N": N, "nc": nc})
    return reqs


def run(S, ctx, reqs, slots, budget=0):
    srv = S.sbio_server_create(ctx, slots, budget)
    outs, tickets, sphs = [], [], []
    for r in reqs:
        op = S.SBIO_OP_LAPLACE if r["op"] == "laplace" else S.SBIO_OP_STOKES
        out = np.zeros((NAPPLY, 2 * r["N"]) if r["op"] == "laplace" else (NAPPLY, r["N"], 3))
        sph = S.make_spheroids(r["s"].kind, r["s"].A, r["s"].C, r["s"].center, r["s"].quat)
        sphs.append(sph)
        outs.append(out)
        tickets.append(S.sbio_server_submit(srv, op, sph, r["p"], r["coef"], out, NAPPLY))
    lat = []
    for t in tickets:
        st, l, svc = S.sbio_server_wait(srv, t, 600.0)
        assert st == 0
        lat.append(l)
    S.sbio_server_destroy(srv)
    return outs, lat


def test_alone_equals_in_the_mix_and_direct_apply(S):
    ctx = S.sbio_ctx_create(0, 0)
    reqs = make_requests()
    alone = [run(S, ctx, [r], 1)[0][0] for r in reqs]
    mixed, lat = run(S, ctx, reqs, 4)
    for a, m in zip(alone, mixed):
        assert np.max(np.abs(a - m)) <= 1e-12 * np.max(np.abs(a))
    # direct applies on a resident geometry give the same numbers
    for r, a in zip(reqs, alone):
        g = S.Geometry(ctx, r["s"], precision=S.SBIO_MIXED)
        for k in range(NAPPLY):
            if r["op"] == "laplace":
                sig = torch.from_numpy(r["coef"][k, 0].copy()).cuda()
                mu = torch.from_numpy(r["coef"][k, 1].copy()).cuda()
                So = torch.empty(g.N, dtype=torch.float64, device="cuda")
                Do = torch.empty_like(So)
                S.sbio_apply_laplace(g.h, sig, mu, So, Do)
                ref = torch.cat([So, Do]).cpu().numpy()
            else:
                f = torch.from_numpy(r["coef"][k].copy()).cuda()
                u = torch.empty((g.N, 3), dtype=torch.float64, device="cuda")
                S.sbio_apply_stokes_sl(g.h, f, u)
                ref = u.cpu().numpy()
            torch.cuda.synchronize()
            assert np.max(np.abs(a[k] - ref)) <= 1e-12 * np.max(np.abs(ref))
        g.close()
    S.sbio_ctx_destroy(ctx)


def test_memory_budget_admission_completes_everything(S):
    ctx = S.sbio_ctx_create(0, 0)
    reqs = make_requests()
    ref, _ = run(S, ctx, reqs, 1)
    # budget smaller than the sum of the requests: admission must wait for memory
    out, lat = run(S, ctx, reqs, 4, budget=12 << 20)
    for a, b in zip(ref, out):
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))
    S.sbio_ctx_destroy(ctx)


def test_invalid_request_rejected(S):
    ctx = S.sbio_ctx_create(0, 0)
    srv = S.sbio_server_create(ctx, 1)
    s = I.rsa_suspension(2, 0.1, 1, 4)
    sph = S.make_spheroids(s.kind, s.A, s.C, s.center, s.quat)
    coef = np.zeros((1, 2, 2, 25))
    out = np.zeros((1, 2 * 2 * 50))
    with pytest.raises(S.SbioError) as e:
        S.sbio_server_submit(srv, 7, sph, 4, coef, out, 1)
    assert e.value.code == S.SBIO_EINVAL
    with pytest.raises(S.SbioError) as e:
        S.sbio_server_wait(srv, 12345, 0.1)
    assert e.value.code == S.SBIO_EINVAL
    S.sbio_server_destroy(srv)
    S.sbio_ctx_destroy(ctx)


def test_served_results_against_oracle_sampled(S):
    """One Laplace S + D and one Stokes request served together (mixed
    precision) against the CPU oracle's method on sampled targets, for every
    apply of each request, at the mixed bound."""
    from oracle import geometry as OG
    from oracle import laplace as OL
    from oracle import stokes as OSt

    ctx = S.sbio_ctx_create(0, 0)
    reqs = [r for r in make_requests() if r["s"].M in (14, 5)]     # one Laplace (M 14, p 8), one Stokes (M 5, p 12)
    assert sorted(r["op"] for r in reqs) == ["laplace", "stokes"]
    outs, _ = run(S, ctx, reqs, 2)
    for k, (r, out) in enumerate(zip(reqs, outs)):
        og = OG.SuspensionGeom.from_suspension(r["s"])
        tg = np.sort(np.random.default_rng(k).choice(r["N"], 25, replace=False))
        for a in range(NAPPLY):
            if r["op"] == "laplace":
                Sr, Dr = OL.LaplaceOracle(og).apply(r["coef"][a, 0], r["coef"][a, 1], "method", targets=tg)
                for got, ref in ((out[a][:r["N"]][tg], Sr), (out[a][r["N"]:][tg], Dr)):
                    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-6
            else:
                Ur = OSt.StokesOracle(og).apply(r["coef"][a], "method", targets=tg)
                assert np.max(np.abs(out[a][tg] - Ur)) / np.max(np.abs(Ur)) < 1e-6
    S.sbio_ctx_destroy(ctx)


def test_treecode_requests_alone_in_mix_and_against_direct(S):
    """A Laplace request with the treecode flag, large enough (67,600 nodes)
    for the server to use it: the same alone and in a mix with direct and
    Stokes requests, and within the treecode bound of the direct-field
    results."""
    ctx = S.sbio_ctx_create(0, 0)
    base = make_requests()
    big = I.rsa_suspension(200, 0.2, 777, 12, name="srvtree")
    nc = 169
    rng = np.random.default_rng(77)
    coef = np.ascontiguousarray(np.stack([I.coefficients(rng, 200, 12, 2).transpose(1, 0, 2) for _ in range(NAPPLY)]))
    N = 200 * 13 * 26
    reqs = base + [{"s": big, "p": 12, "op": "laplace", "coef": coef, "N": N, "nc": nc}]

    def run_flags(rs, slots, tree_for):
        srv = S.sbio_server_create(ctx, slots, 0)
        outs, tickets, keep = [], [], []
        for r in rs:
            op = S.SBIO_OP_LAPLACE if r["op"] == "laplace" else S.SBIO_OP_STOKES
            out = np.zeros((NAPPLY, 2 * r["N"]) if r["op"] == "laplace" else (NAPPLY, r["N"], 3))
            sph = S.make_spheroids(r["s"].kind, r["s"].A, r["s"].C, r["s"].center, r["s"].quat)
            keep.append(sph)
            outs.append(out)
            fl = S.SBIO_REQ_TREE if r is tree_for else 0
            tickets.append(S.sbio_server_submit(srv, op, sph, r["p"], r["coef"], out, NAPPLY, flags=fl))
        for t in tickets:
            st, _, _ = S.sbio_server_wait(srv, t, 600.0)
            assert st == 0
        S.sbio_server_destroy(srv)
        return outs

    tree_req = reqs[-1]
    alone = run_flags([tree_req], 1, tree_req)[0]
    mixed = run_flags(reqs, 4, tree_req)[-1]
    direct = run_flags([tree_req], 1, None)[0]
    assert np.max(np.abs(alone - mixed)) <= 1e-12 * np.max(np.abs(alone))
    for a in range(NAPPLY):
        for part in (slice(0, N), slice(N, 2 * N)):
            ref = direct[a][part]
            assert np.max(np.abs(alone[a][part] - ref)) / np.max(np.abs(ref)) < 1e-6
    S.sbio_ctx_destroy(ctx)
