"""GPU parity of the whole step (through the C-ABI) against the FP64 oracle.

Sizes are chosen so the oracle finishes in seconds while the kernels still run over
several tiles, cells and blocks with ragged tails (point counts that are not multiples of
32 or 256, levels of 1 and 2 vertices per axis, grids of up to 64^3)."""
import numpy as np
import pytest

from oracle import pdg_oracle as O
from paper_2509_18097_gb300 import synth
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def rng(s):
    return np.random.Generator(np.random.PCG64(s))


def small_sphere(seed=0, n_src=701, n_tgt=903, res=(4, 8, 16), sub=2, amp=0.1, theta_sigma=0.02):
    r = rng(seed)
    v, _, e = synth.icosphere(sub)
    src = synth.sphere_points(r, n_src).astype(np.float32)
    tgt = synth.sinusoid(synth.sphere_points(r, n_tgt), amp).astype(np.float32)
    th = [(r.standard_normal((n, n, n, 3)) * theta_sigma).astype(np.float32) for n in res] if theta_sigma else None
    return synth.Workload("small_sphere", v, e, src, tgt, tuple(res), thetas=th)


def mid_ellipsoid(seed=1):
    r = rng(seed)
    axes = (1.0, 0.7, 0.5)
    v, _, e = synth.geodesic_sphere(20, axes)
    src = synth.ellipsoid_points(r, 9001, axes).astype(np.float32)
    tgt = synth.sinusoid(synth.ellipsoid_points(r, 11003, axes), 0.05).astype(np.float32)
    res = (8, 16, 32, 64)
    th = [(r.standard_normal((n, n, n, 3)) * 0.01).astype(np.float32) for n in res]
    return synth.Workload("mid_ellipsoid", v, e, src, tgt, res, thetas=th)


CASES = {
    "small": lambda: small_sphere(),
    "levels_1_2": lambda: small_sphere(seed=3, res=(1, 2, 32), n_src=257, n_tgt=1000),
    "single_pair_zero_grids": lambda: synth.single_pair(),
    "mid": mid_ellipsoid,
}


@pytest.mark.parametrize("case", list(CASES))
def test_one_step_stagewise(case):
    w = CASES[case]()
    g = H.gpu_run(w, thetas=w.thetas)
    info = H.stagewise(w, g, H.oracle_cfg(w))
    print(case, info)


def test_one_step_stagewise_headline():
    """The headline workload at full size (50 412 vertices, 100k + 100k points,
    16^3..128^3, grids N(0, 0.01^2)): every stage of one step against the oracle."""
    w = synth.ellipsoid_pair(seed=0)
    g = H.gpu_run(w, thetas=w.thetas)
    info = H.stagewise(w, g, H.oracle_cfg(w))
    print("headline", info)


@pytest.mark.parametrize("variant", [dict(precondition=False), dict(robust_weight_stopgrad=True),
                                     dict(w_iso=0.0, w_chamfer_mesh=2.0, w_chamfer_pts=0.5)])
def test_one_step_config_variants(variant):
    w = small_sphere(seed=5)
    g = H.gpu_run(w, cfg_kwargs=variant, thetas=w.thetas)
    H.stagewise(w, g, H.oracle_cfg(w, **variant))


def test_one_step_end_to_end_losses_and_positions():
    """GPU and oracle each run the step from the same state; losses and the updated
    positions agree (no stage fed from the other side)."""
    w = small_sphere(seed=7)
    g = H.gpu_run(w, thetas=w.thetas)
    cfg = H.oracle_cfg(w)
    st = O.begin_frame(w.template, w.source, w.target, w.edges, cfg, [t.astype(np.float64) for t in w.thetas])
    o = O.step(st, cfg)
    H.check_close("loss", g["loss"], [o["loss"], o["cd_mesh"], o["cd_pts"], o["iso"]])
    H.check_close("y", g["y"], o["y"])
    Xo, _ = O.end_frame(st, cfg)
    H.check_close("X_t after one step", g["verts"], Xo)


def test_trajectory_single_pair_20_steps():
    """Config single_pair (642 verts, 2048 + 2048 points, 8^3/16^3/32^3), 20 free-running
    steps on each side: final vertex positions and the last losses agree."""
    w = synth.single_pair()
    steps = 20
    g = H.gpu_run(w, steps=steps, read=False)
    cfg = H.oracle_cfg(w)
    X, hist, st = O.fit_frame(w.template, w.source, w.target, w.edges, cfg, steps)
    s = g["stats"]
    H.check_close("last losses", [s.loss_total, s.cd_mesh, s.cd_pts, s.iso], hist[-1], rtol=1e-4)
    H.check_close("X_t", g["verts"], X, rtol=1e-4, atol_rel=1e-5)


def test_deterministic_bitwise():
    w = small_sphere(seed=9)
    a = H.gpu_run(w, thetas=w.thetas, steps=3)
    b = H.gpu_run(w, thetas=w.thetas, steps=3)
    for k in ("y", "g_pts", "nn_fwd", "nn_rev", "loss"):
        assert np.array_equal(a[k], b[k]), k
    for l in range(len(w.res)):
        assert np.array_equal(a["grads"][l], b["grads"][l])
        assert np.array_equal(a["theta1"][l], b["theta1"][l])
    assert np.array_equal(a["verts"], b["verts"])


def test_exact_ties_lowest_index():
    """Duplicated target points (exact ties) resolve to the lowest index on the GPU."""
    r = rng(11)
    v, _, e = synth.icosphere(1)
    base = synth.sphere_points(r, 300)
    tgt = np.concatenate([base, base, base[:100]]).astype(np.float32)  # triplicates
    src = base[:250].astype(np.float32)  # queries coincide with target points (d2 = 0 ties)
    w = synth.Workload("ties", v, e, src, tgt, (4, 8))
    g = H.gpu_run(w)
    V = len(v)
    idx, _ = O.nn_bruteforce(g["y"][V:].astype(np.float64), tgt.astype(np.float64))
    assert np.array_equal(g["nn_fwd"][V:], idx)
    assert np.all(g["nn_fwd"][V:] < 300)


def test_outlier_queries_use_the_ring_search():
    """Template vertices far from a small target cloud need rings beyond the first
    (and the exhaustive fallback); their neighbours are still exact."""
    r = rng(12)
    v, _, e = synth.icosphere(2)
    tgt = (synth.sphere_points(r, 200) * 0.2 + np.array([1.0, 0.5, 0.0])).astype(np.float32)
    src = synth.sphere_points(r, 400).astype(np.float32)
    w = synth.Workload("outliers", v, e, src, tgt, (4, 16))
    g = H.gpu_run(w)
    V = len(v)
    y = g["y"].astype(np.float64)
    H.nn_check("fwd", g["nn_fwd"], y, tgt.astype(np.float64))
    H.nn_check("rev X", g["nn_rev"][0], tgt.astype(np.float64), y[:V])


def test_step_graph_kernel_count():
    """One step of levels up to 128^3 is 15 launches: interpolation (which also starts the
    step's Adam count), two scan phases and the scatter of the moving grid, the two NN passes,
    isometry, assembly, the two loss kernels, adjoint, the three preconditioner passes and
    Adam.  The plan's item prefixes are computed outside the step, once per frame."""
    g = H.gpu_run(small_sphere(seed=13), read=False)
    assert g["kernels_per_step"] == 15
