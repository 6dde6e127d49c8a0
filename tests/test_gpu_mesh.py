"""GPU parity of the template-mesh fit (Sec. 3.4, surface initialisation loss
L_mesh = CD_R(X_0, P_0); Sec. 3.6, lambda = 16, lr = 1e-4) against the FP64 oracle.

One iteration is checked stage by stage, each stage on the GPU's own input: the vertex
gradient of the robust Chamfer loss, the preconditioned gradient (I + lambda L)^{-2} g, and
Adam's first step.  A 30-iteration fit is compared free-running with the oracle's.

Tolerance of the preconditioned gradient: two FP32 Chebyshev solves of ~135 three-term
iterations each (lambda = 16, max degree 6: the interval [1, 193]).  A float32 emulation of
the recurrence on icospheres of 162 to 2562 vertices, against the sparse direct solve,
stays within 1.1e-6 of max|result| for Chamfer gradients and random right-hand sides; the
test allows 1e-5 of max|result| plus the usual 1e-5 relative.

Tolerance of the free-running fit: each Adam step moves a coordinate by about lr in the
direction of the sign of its preconditioned gradient, so a coordinate whose gradient is
within rounding of zero can step the other way (a departure of up to 2 lr there); FP64 runs
with 1e-6 relative noise on the preconditioned gradient and FP32 rounding of the vertices
stay within 0.2 lr of the exact run after 30 iterations, on under 1% of the coordinates,
with the loss within 1e-6 relative.  The test allows 2 lr on any coordinate, 1e-6 on all
but 2% of them, and 1e-5 relative on the loss.
"""
import numpy as np
import pytest

from oracle import pdg_oracle as O
from paper_2509_18097_gb300 import synth
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

LAM, LR = O.MESH_LAMBDA, O.MESH_LR


def rng(s):
    return np.random.Generator(np.random.PCG64(s))


def sphere_fit_case(seed, subdiv=3, n_p0=1003):
    """Icosphere template against a sinusoid-deformed sphere inflated by 5% (ragged cloud)."""
    r = rng(seed)
    v, _, e = synth.icosphere(subdiv)
    p0 = synth.sinusoid(synth.sphere_points(r, n_p0) * 1.05, 0.05).astype(np.float32)
    return v.astype(np.float32), e, p0


def make_ctx(B, v, e, p0, res=(4, 8)):
    cfg = B.pdg_config_default(res=res, lo=(-1.5,) * 3, hi=(1.5,) * 3)
    return B.pdg_create(cfg, v, e, p0, max_pts=len(p0))


def fit(v, e, p0, n_steps, lam=LAM, lr=LR, res=(4, 8)):
    """Runs the fit through the C-ABI; returns the fitted vertices, gradient, preconditioned
    gradient (of the last iteration) and the stats."""
    import torch

    from paper_2509_18097_gb300 import binding as B

    ctx = make_ctx(B, v, e, p0, res)
    try:
        st = B.pdg_fit_mesh(ctx, p0, n_steps, lam, lr)
        torch.cuda.synchronize()
        V = len(v)
        out = dict(stats=st, X=B.pdg_get_vertices(ctx, np.empty((V, 3), np.float32)))
        if n_steps > 0:
            out["grad"] = B.pdg_read(ctx, B.BUF_MESH_GRAD, 0, np.empty((V, 3), np.float32))
            out["pgrad"] = B.pdg_read(ctx, B.BUF_MESH_PGRAD, 0, np.empty((V, 3), np.float32))
        return out
    finally:
        B.pdg_destroy(ctx)


def tie_excluded(X, P):
    """Vertices whose gradient involves a nearest-neighbour near-tie (either direction): the
    two candidates of a near-tied reverse query, the vertex of a near-tied forward query."""
    from scipy.spatial import cKDTree

    excl = np.zeros(len(X), bool)
    idx, d2 = O.nn_exact(X, P)
    excl |= O.nn_second_gap(X, P, idx, d2) < H.NEAR_TIE
    ridx, rd2 = O.nn_exact(P, X)
    near = O.nn_second_gap(P, X, ridx, rd2) < H.NEAR_TIE
    if near.any():
        _, cand = cKDTree(X).query(P[near], k=2)
        excl[cand.ravel()] = True
    return excl


def check_one_step(v, e, p0, lam=LAM, lr=LR):
    g = fit(v, e, p0, 1, lam, lr)
    X0 = v.astype(np.float64)
    P = p0.astype(np.float64)
    ch = O.robust_chamfer(X0, P)
    excl = tie_excluded(X0, P)
    # the loss is continuous at a tie: compared whatever the tie count
    H.check_close("L_mesh", [g["stats"].cd_mesh, g["stats"].loss_total], [ch["loss"], ch["loss"]])
    H.check_close("dL/dX", g["grad"], ch["grad_A"], mask=~excl)
    pg_ref = O.mesh_precondition(g["grad"].astype(np.float64), e, lam)
    H.check_close("(I + lam L)^-2 g", g["pgrad"], pg_ref, atol_rel=1e-5)
    x1, _, _ = O.adam_update(X0, 0.0, 0.0, g["pgrad"].astype(np.float64), 1, lr)
    H.check_close("X_1", g["X"], x1)
    return dict(excluded=int(excl.sum()), grad=g["grad"], pgrad=g["pgrad"])


@pytest.mark.parametrize("subdiv,n_p0", [(2, 257), (3, 1003), (4, 5000)])
def test_mesh_fit_one_step_stagewise(subdiv, n_p0):
    v, e, p0 = sphere_fit_case(60 + subdiv, subdiv, n_p0)
    info = check_one_step(v, e, p0)
    print("mesh one step", subdiv, n_p0, info["excluded"])


def test_mesh_fit_one_step_headline():
    """The 50 412-vertex geodesic ellipsoid fitted to its 100k-point keyframe cloud."""
    w = synth.ellipsoid_pair(seed=0, theta_sigma=0)
    info = check_one_step(w.template.astype(np.float32), w.edges, w.source)
    print("mesh headline", info["excluded"])


def test_mesh_fit_lambda_zero_is_the_raw_gradient():
    """lambda = 0: A = I, the solves return their right-hand side exactly."""
    v, e, p0 = sphere_fit_case(64)
    g = fit(v, e, p0, 1, lam=0.0)
    np.testing.assert_array_equal(g["pgrad"], g["grad"])


def test_mesh_fit_trajectory_30_steps():
    v, e, p0 = sphere_fit_case(65, 4, 8000)
    K = 30
    g = fit(v, e, p0, K)
    st = O.mesh_begin(v.astype(np.float64), p0.astype(np.float64), e)
    losses = [O.mesh_step(st)["loss"] for _ in range(K)]
    assert losses[-1] < losses[0]
    H.check_close("L_mesh after 29 updates", [g["stats"].cd_mesh], [losses[-1]], rtol=1e-5)
    d = np.abs(g["X"].astype(np.float64) - st.X)
    far = d > 1e-6
    print("mesh trajectory: max |dX| / lr", d.max() / LR, "coordinates past 1e-6:", int(far.sum()), "of", d.size)
    assert d.max() <= 2 * LR, d.max() / LR
    assert far.mean() <= 0.02, far.mean()
    assert g["stats"].n_steps == K and g["stats"].status == 0


def test_mesh_fit_feeds_the_next_frame_and_state_rules():
    """The fitted vertices are the template the next frame starts from (zero grids: y = X);
    the fit is refused inside a frame and its buffers are unreadable once a frame began."""
    import torch

    from paper_2509_18097_gb300 import binding as B

    v, e, p0 = sphere_fit_case(66)
    V = len(v)
    ctx = make_ctx(B, v, e, p0)
    try:
        with pytest.raises(B.PdgError) as ei:
            B.pdg_read(ctx, B.BUF_MESH_GRAD, 0, np.empty((V, 3), np.float32))
        assert ei.value.status == B.ERR_STATE
        st = B.pdg_fit_mesh(ctx, p0, 0)  # no iterations: nothing moves
        assert st.n_steps == 0
        np.testing.assert_array_equal(B.pdg_get_vertices(ctx, np.empty((V, 3), np.float32)), v)
        B.pdg_fit_mesh(ctx, p0, 5)
        X = B.pdg_get_vertices(ctx, np.empty((V, 3), np.float32))
        assert np.abs(X - v).max() > 0
        B.pdg_read(ctx, B.BUF_MESH_PGRAD, 0, np.empty((V, 3), np.float32))
        B.pdg_begin_frame(ctx, p0)
        with pytest.raises(B.PdgError) as ei:
            B.pdg_fit_mesh(ctx, p0, 1)
        assert ei.value.status == B.ERR_STATE
        with pytest.raises(B.PdgError) as ei:
            B.pdg_read(ctx, B.BUF_MESH_GRAD, 0, np.empty((V, 3), np.float32))
        assert ei.value.status == B.ERR_STATE
        B.pdg_step(ctx, 1)
        torch.cuda.synchronize()
        y = B.pdg_read(ctx, B.BUF_Y, 0, np.empty((V + len(p0), 3), np.float32))
        np.testing.assert_array_equal(y[:V], X)
        B.pdg_end_frame(ctx)
    finally:
        B.pdg_destroy(ctx)


def test_mesh_fit_rejections():
    from paper_2509_18097_gb300 import binding as B

    v, e, p0 = sphere_fit_case(67)
    ctx = make_ctx(B, v, e, p0)
    try:
        for args, code in (((np.concatenate([p0, p0]), 1), B.ERR_BUDGET), ((p0, -1), B.ERR_INVALID),
                           ((p0, 1, float("nan")), B.ERR_INVALID), ((p0, 1, LAM, -1.0), B.ERR_INVALID),
                           ((p0, 1, 1e5 / 6 + 1.0), B.ERR_INVALID)):  # icosphere: degree 6 at most
            with pytest.raises(B.PdgError) as ei:
                B.pdg_fit_mesh(ctx, *args)
            assert ei.value.status == code
        np.testing.assert_array_equal(B.pdg_get_vertices(ctx, np.empty((len(v), 3), np.float32)), v)
    finally:
        B.pdg_destroy(ctx)
