"""GPU parity at level resolutions with a factor 3 (2^a 3^b vertices per axis, odd sizes
included): those levels take the tile path of the preconditioner, whose line transforms are
mixed radix-2/3 Stockham FFTs.

Pins: a product of DCT-II cosine modes is an eigenvector of the free-boundary grid
Laplacian with eigenvalue sum 4 sin^2(pi k / 2n) (Sec. 3.2, Eq. 3), so the preconditioner
scales it by the closed form (1 + lambda mu)^{-2}; one step stage by stage against the
oracle on pyramids such as 6/12/24/48, 3/9/27/81 and 54/108/216; a batch mixing both paths
bitwise equal to each member run alone.

Tolerance of the closed-form check: the four line transforms of the tile path each add
O(log2 n * 6e-8) of the input's norm, so the bound is 1e-6 of max|g| plus 1e-5 relative."""
import numpy as np
import pytest

from tests import gpu_helpers as H
from tests.test_gpu_batch import job, make, snapshot, solo
from tests.test_gpu_parity import small_sphere

pytestmark = pytest.mark.gpu


def cosine_mode(n, k):
    """prod_a cos(pi k_a (i_a + 1/2) / n) on the [z, y, x] vertex grid; k = (kz, ky, kx)."""
    c = [np.cos(np.pi * ka * (np.arange(n) + 0.5) / n) for ka in k]
    return c[0][:, None, None] * c[1][None, :, None] * c[2][None, None, :]


def mode_eigenvalue(n, k):
    return sum(4.0 * np.sin(np.pi * ka / (2.0 * n)) ** 2 for ka in k)


@pytest.mark.parametrize("n", [3, 6, 9, 24, 27, 48, 81, 96, 162, 192, 216])
def test_precondition_cosine_modes_closed_form(n):
    from paper_2509_18097_gb300 import binding as B

    w = small_sphere(seed=40, theta_sigma=0)
    lam = 1.75
    cfg = B.pdg_config_default(res=(n,), lambda0=lam)
    ctx = B.pdg_create(cfg, w.template, w.edges, w.source, max_pts=max(len(w.source), len(w.target)))
    try:
        ks = [(1, 0, 0), (n - 1, n // 2, min(3, n - 1)), (n // 3, min(2, n - 1), n - 2 if n > 2 else 1)]
        g = np.stack([cosine_mode(n, k).ravel() * s for k, s in zip(ks, (1.0, -2.0, 0.5))], -1).astype(np.float32)
        out = B.pdg_precondition(ctx, 0, g, np.empty_like(g))
        ref = np.stack([g[:, c].astype(np.float64) * (1.0 + lam * mode_eigenvalue(n, k)) ** -2
                        for c, k in enumerate(ks)], -1)
        for c in range(3):
            H.check_close(f"n={n} mode {ks[c]}", out[:, c], ref[:, c], terms=np.abs(g[:, c]).max())
    finally:
        B.pdg_destroy(ctx)


@pytest.mark.parametrize("res", [(6, 12, 24, 48), (3, 9, 27, 81), (16, 48, 96), (54, 108, 216)])
def test_one_step_stagewise_mixed_radix(res):
    """One step from random grids on every level: every stage against the oracle, the
    preconditioned gradient of the tile path and Adam fused into its last pass included."""
    w = small_sphere(seed=41, n_src=1501, n_tgt=1203, res=res, theta_sigma=0.01)
    g = H.gpu_run(w, thetas=w.thetas)
    info = H.stagewise(w, g, H.oracle_cfg(w))
    print("mixed radix", res, info)


def test_batch_with_mixed_radix_members_matches_solo_bitwise():
    from paper_2509_18097_gb300 import binding as B

    jobs = [job(5, res=(6, 24, 48)), job(6, sub=3, n_src=2000, n_tgt=900, res=(8, 16, 32, 64)),
            job(7, res=(4, 12, 36, 144))]
    steps = 3
    ref = [solo(B, w, steps) for w in jobs]
    ctxs = [make(B, w) for w in jobs]
    b = B.pdg_batch_create(4)
    try:
        B.pdg_batch_set(b, ctxs)
        B.pdg_batch_step(b, steps)
        for w, c, r in zip(jobs, ctxs, ref):
            s = snapshot(B, c, w)
            for k in r:
                assert np.array_equal(s[k], r[k]), (w.name, k)
    finally:
        for c in ctxs:
            B.pdg_destroy(c)
        B.pdg_batch_destroy(b)
