"""The GPU Sobolev preconditioner (pdg_precondition, the same kernels as the step) against
the closed form on DCT-II cosine modes at every supported resolution, including the 256^3
tile path, and against the oracle's CG solve on random gradients."""
import math

import numpy as np
import pytest

from oracle import pdg_oracle as O
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def ctx_for(B, n, lam0=0.25):
    v = np.zeros((1, 3), np.float32)
    cfg = B.pdg_config_default(res=(n,), lambda0=lam0)
    return B.pdg_create(cfg, v, np.zeros((0, 2), np.int32), v, max_pts=1)


def mode(n, k):
    i = (np.arange(n, dtype=np.float64) + 0.5) * np.pi / n
    cx, cy, cz = np.cos(k[0] * i), np.cos(k[1] * i), np.cos(k[2] * i)
    return (cz[:, None, None] * cy[None, :, None] * cx[None, None, :]).reshape(-1)


def factor(n, k, lam):
    mu = sum(4 * math.sin(math.pi * kd / (2 * n)) ** 2 for kd in k)
    return (1 + lam * mu) ** -2


@pytest.mark.parametrize("n", [2, 4, 8, 16, 32, 64, 128, 256])
def test_cosine_modes_scale_by_closed_form(n):
    from paper_2509_18097_gb300 import binding as B

    lam = 0.6
    ks = [(0, 0, 0), (1, 0, min(3, n - 1)), (n - 1, n // 2, 1), (n // 3, n - 1, n - 1)]
    g = np.zeros((n**3, 3), np.float64)
    exp = np.zeros_like(g)
    for c in range(3):
        for j, k in enumerate(ks):
            a = (1.0 + j + c) * (-1) ** j
            m = mode(n, k)
            g[:, c] += a * m
            exp[:, c] += a * factor(n, k, lam) * m
    ctx = ctx_for(B, n, lam0=lam)
    try:
        out = B.pdg_precondition(ctx, 0, g.astype(np.float32), np.empty((n**3, 3), np.float32))
    finally:
        B.pdg_destroy(ctx)
    H.check_close(f"modes n={n}", out, exp)


@pytest.mark.parametrize("n", [64, 128])
def test_cosine_modes_with_slowly_converging_pivots(n):
    """lambda = 8: the z-solve pivots reach their FP32 limit only after about 28 rows, so
    the solves read every pivot from the table instead of holding 16 plus the limit in
    registers; the result must be the same closed form."""
    from paper_2509_18097_gb300 import binding as B

    lam = 8.0
    ks = [(0, 0, 0), (1, 2, 0), (0, 0, 1), (n // 2, 1, n - 1), (3, n - 1, 5)]
    g = np.zeros((n**3, 3), np.float64)
    exp = np.zeros_like(g)
    for c in range(3):
        for j, k in enumerate(ks):
            a = (1.0 + j + c) * (-1) ** j
            m = mode(n, k)
            g[:, c] += a * m
            exp[:, c] += a * factor(n, k, lam) * m
    ctx = ctx_for(B, n, lam0=lam)
    try:
        out = B.pdg_precondition(ctx, 0, g.astype(np.float32), np.empty((n**3, 3), np.float32))
    finally:
        B.pdg_destroy(ctx)
    H.check_close(f"modes lambda=8 n={n}", out, exp)


@pytest.mark.parametrize("n", [4, 16, 32])
def test_random_gradient_matches_oracle_cg(n):
    from paper_2509_18097_gb300 import binding as B

    r = np.random.Generator(np.random.PCG64(n))
    g = r.standard_normal((n**3, 3)).astype(np.float32)
    g[r.random(n**3) < 0.7] = 0.0  # sparse, like gradients near the data only
    ctx = ctx_for(B, n, lam0=0.84375)
    try:
        out = B.pdg_precondition(ctx, 0, g, np.empty_like(g))
    finally:
        B.pdg_destroy(ctx)
    ref = O.sobolev_precondition(g.reshape(n, n, n, 3).astype(np.float64), 0.84375).reshape(-1, 3)
    H.check_close(f"random n={n}", out, ref)


def test_precondition_is_refused_inside_a_frame():
    from paper_2509_18097_gb300 import binding as B

    ctx = ctx_for(B, 4)
    B.pdg_begin_frame(ctx, np.zeros((1, 3), np.float32))
    with pytest.raises(B.PdgError) as e:
        B.pdg_precondition(ctx, 0, np.zeros((64, 3), np.float32), np.empty((64, 3), np.float32))
    assert e.value.status == B.ERR_STATE
    B.pdg_end_frame(ctx)
    B.pdg_destroy(ctx)
