"""Writes tests/golden/tiny_laplace.json from the CPU oracle only.

Case: one prolate (A=0.6, C=1.4) and one oblate (A=1.2, C=0.45) spheroid,
p = 4, near factor 2 (so both near and far branches occur), fixed
coefficients; expected S and D at every node by the oracle's method mode
(and its exact mode, for the record).  Re-run after a change to the oracle's
arithmetic that a cited passage justifies.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import geometry as OG  # noqa: E402
from oracle import laplace as OL  # noqa: E402

CASE = {
    "kind": [0, 1],
    "A": [0.6, 1.2],
    "C": [1.4, 0.45],
    "center": [[0.0, 0.0, 0.0], [3.6, 0.4, -0.3]],
    "quat": [[1.0, 0.0, 0.0, 0.0], [0.8, 0.2, -0.5, 0.26]],
    "p": 4,
    "near_factor": 2.0,
}


def coefficients(p, M, salt):
    nc = (p + 1) ** 2
    k = np.arange(nc)
    n = np.floor(np.sqrt(k))
    c = np.array([[np.cos(1.3 * kk + 0.7 * i + salt) for kk in k] for i in range(M)])
    return c / (n + 1.0) ** 2


def main():
    q = np.array(CASE["quat"])
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    g = OG.SuspensionGeom(np.array(CASE["kind"]), np.array(CASE["A"]), np.array(CASE["C"]),
                          np.array(CASE["center"]), q, CASE["p"], near_factor=CASE["near_factor"])
    sig = coefficients(CASE["p"], 2, 0.0)
    mu = coefficients(CASE["p"], 2, 1.0)
    O = OL.LaplaceOracle(g)
    S, D = O.apply(sig, mu, "method")
    Se, De = O.apply(sig, mu, "exact")
    out = dict(CASE, quat=q.tolist(), sigma_tilde=sig.tolist(), mu_hat=mu.tolist(), S_method=S.tolist(),
               D_method=D.tolist(), S_exact=Se.tolist(), D_exact=De.tolist(),
               near_pairs=int(g.near_matrix().sum()))
    with open(os.path.join(HERE, "tiny_laplace.json"), "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    main()
