"""The mixed near form runs the Ferrers functions normalised, by a
three-term recurrence whose constants are closed forms (the host table of
the kernel, documented beside it):
    Pbar_0^0 = 1/sqrt(4 pi),  Pbar_1^1 = sqrt(3) sv Pbar_0^0,
    Pbar_m^m = sqrt((2m+1)/(2m)) sv Pbar_{m-1}^{m-1}  (m >= 2),
    Pbar_n^m = a_nm v Pbar_{n-1}^m - b_nm Pbar_{n-2}^m,
    a_nm = sqrt((2n+1)(2n-1)/((n-m)(n+m))),
    b_nm = sqrt((2n+1)(n+m-1)(n-m-1)/((2n-3)(n-m)(n+m))).
Pinned here against the oracle's (scipy-pinned) Ferrers functions times
the surface-harmonic normalisation sqrt(2)^[m != 0] N_n^m, in FP64 and run
in FP32 (the kernel's precision) at the bound the FP32 recurrence keeps."""
import math

import numpy as np

from oracle import legendre as L


def _recurrence(v, N, dtype):
    v = np.asarray(v, dtype=dtype)
    sv = np.sqrt(np.maximum(dtype(1) - v * v, dtype(0))).astype(dtype)
    out = np.zeros(v.shape + (N + 1, N + 1), dtype=dtype)
    pmm = np.full(v.shape, 1.0 / math.sqrt(4.0 * math.pi), dtype=dtype)
    for m in range(N + 1):
        if m == 1:
            pmm = (pmm * dtype(math.sqrt(3.0)) * sv).astype(dtype)
        elif m >= 2:
            pmm = (pmm * dtype(math.sqrt((2.0 * m + 1.0) / (2.0 * m))) * sv).astype(dtype)
        prev, cur = np.zeros_like(pmm), pmm
        out[..., m, m] = cur
        for n in range(m + 1, N + 1):
            a = dtype(math.sqrt((2.0 * n + 1.0) * (2.0 * n - 1.0) / ((n - m) * (n + m))))
            b = dtype(math.sqrt((2.0 * n + 1.0) * (n + m - 1.0) * (n - m - 1.0) / ((2.0 * n - 3.0) * (n - m) * (n + m)))
                      if n >= m + 2 else 0.0)
            nxt = (a * v * cur - b * prev).astype(dtype)
            prev, cur = cur, nxt
            out[..., n, m] = cur
    return out


def _reference(v, N):
    P = L.ferrers_P(v, N)
    ref = np.zeros_like(P)
    for n in range(N + 1):
        for m in range(n + 1):
            ref[..., n, m] = (math.sqrt(2.0) if m else 1.0) * L.norm_factor(n, m) * P[..., n, m]
    return ref


def test_normalised_ferrers_constants_fp64():
    v = np.concatenate([np.linspace(-1.0, 1.0, 41), np.random.default_rng(3).uniform(-1, 1, 200)])
    N = 24
    got, ref = _recurrence(v, N, np.float64), _reference(v, N)
    scale = np.max(np.abs(ref), axis=0, keepdims=True) + 1e-300
    assert np.max(np.abs(got - ref) / scale) < 1e-13


def test_normalised_ferrers_recurrence_in_fp32():
    """The FP32 recurrence stays within about 30 FP32 ulps of the largest
    value of each (n, m) column up to n = 24 (3.8e-6 measured; the forward
    recurrence of the Ferrers functions is stable on [-1, 1]); the near sum
    weights the high orders down, so the near part's error is far smaller
    (1-2e-7 of the largest near value on the GPU)."""
    v = np.random.default_rng(4).uniform(-1, 1, 400)
    N = 24
    got = _recurrence(v.astype(np.float32), N, np.float32).astype(np.float64)
    ref = _reference(v.astype(np.float32).astype(np.float64), N)
    scale = np.max(np.abs(ref), axis=0, keepdims=True) + 1e-300
    err = np.max(np.abs(got - ref) / scale)
    assert err < 1e-5, err
    # the orders of the headline workload (p = 16) at the emulation's level
    err16 = np.max((np.abs(got - ref) / scale)[..., :17, :17])
    assert err16 < 5e-6, err16
