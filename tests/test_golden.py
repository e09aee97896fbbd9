"""Stored oracle values for a tiny two-spheroid case (tests/golden/)."""
import json
import os

import numpy as np
import pytest

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load():
    with open(os.path.join(HERE, "tiny_laplace.json")) as f:
        return json.load(f)


def test_oracle_reproduces_stored_values():
    from oracle import geometry as OG
    from oracle import laplace as OL

    d = load()
    g = OG.SuspensionGeom(np.array(d["kind"]), np.array(d["A"]), np.array(d["C"]), np.array(d["center"]),
                          np.array(d["quat"]), d["p"], near_factor=d["near_factor"])
    S, D = OL.LaplaceOracle(g).apply(np.array(d["sigma_tilde"]), np.array(d["mu_hat"]), "method")
    np.testing.assert_allclose(S, d["S_method"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(D, d["D_method"], rtol=0, atol=1e-13)
    assert int(g.near_matrix().sum()) == d["near_pairs"] > 0
    # method vs exact: the far-quadrature error of the method at p = 4
    assert OL.normwise_rel_err(S, d["S_exact"]) < 1e-2


@pytest.mark.gpu
def test_gpu_matches_stored_values():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as G

    G.build()
    import paper_2506_20809_gb300.sbio as S

    d = load()
    ctx = S.sbio_ctx_create(0, 0)
    sph = S.make_spheroids(d["kind"], d["A"], d["C"], d["center"], d["quat"])
    g = S.sbio_geom_create(ctx, sph, d["p"], near_factor=d["near_factor"])
    info = S.sbio_geom_info(g)
    assert info["n_near_pairs"] == d["near_pairs"]
    sig = torch.tensor(d["sigma_tilde"], dtype=torch.float64, device="cuda")
    mu = torch.tensor(d["mu_hat"], dtype=torch.float64, device="cuda")
    So = torch.empty(info["n_targets"], dtype=torch.float64, device="cuda")
    Do = torch.empty_like(So)
    S.sbio_apply_laplace(g, sig, mu, So, Do)
    torch.cuda.synchronize()
    ref_S, ref_D = np.array(d["S_method"]), np.array(d["D_method"])
    assert np.max(np.abs(So.cpu().numpy() - ref_S)) / np.max(np.abs(ref_S)) < 1e-10
    assert np.max(np.abs(Do.cpu().numpy() - ref_D)) / np.max(np.abs(ref_D)) < 1e-10
    S.sbio_geom_destroy(g)
    S.sbio_ctx_destroy(ctx)
