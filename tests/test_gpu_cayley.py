"""GPU parity of the step with the 6-D Cayley payload of Sec. 3.3 (each grid vertex holds
z and t; a point moves to R(z) x + t with R(z) = (I + Z)(I - Z)^{-1}) against the FP64 oracle:
every stage of one step from random grids, at small, ragged and headline sizes, the frame
end X_t = M(T_t(X_{t-1})) X_{t-1}, and bitwise equality alone and in a batch beside
displacement-payload jobs."""
import numpy as np
import pytest

from oracle import pdg_oracle as O
from paper_2509_18097_gb300 import synth
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

CAYLEY = dict(payload="cayley")


def rng(s):
    return np.random.Generator(np.random.PCG64(s))


def grids6(r, res, z_sigma=0.03, t_sigma=0.01):
    return [np.concatenate([r.standard_normal((n, n, n, 3)) * z_sigma, r.standard_normal((n, n, n, 3)) * t_sigma],
                           -1).astype(np.float32) for n in res]


def sphere_case(seed, n_src=701, n_tgt=903, res=(4, 8, 16), sub=2):
    r = rng(seed)
    v, _, e = synth.icosphere(sub)
    src = synth.sphere_points(r, n_src).astype(np.float32)
    tgt = synth.sinusoid(synth.sphere_points(r, n_tgt), 0.1).astype(np.float32)
    return synth.Workload("cayley_sphere", v, e, src, tgt, tuple(res), thetas=grids6(r, res))


@pytest.mark.parametrize("case", ["small", "levels_1_2", "zero_grids"])
def test_cayley_one_step_stagewise(case):
    if case == "small":
        w = sphere_case(51)
    elif case == "levels_1_2":
        w = sphere_case(52, n_src=257, n_tgt=1000, res=(1, 2, 32))
    else:
        w = sphere_case(53)
        w.thetas = None  # zero grids: the identity, then the first update
    g = H.gpu_run(w, cfg_kwargs=CAYLEY, thetas=w.thetas)
    info = H.stagewise(w, g, H.oracle_cfg(w, payload="cayley"))
    print("cayley", case, info)


def test_cayley_one_step_stagewise_headline():
    """The headline workload (50 412 vertices, 100k + 100k points, 16^3..128^3) with the 6-D
    payload: random z ~ N(0, 0.01^2), t ~ N(0, 0.005^2) on every level."""
    w = synth.ellipsoid_pair(seed=0, theta_sigma=0)
    w.thetas = grids6(rng(54), w.res, 0.01, 0.005)
    g = H.gpu_run(w, cfg_kwargs=CAYLEY, thetas=w.thetas)
    info = H.stagewise(w, g, H.oracle_cfg(w, payload="cayley"))
    print("cayley headline", info)


def test_cayley_frame_end_and_second_frame():
    """After a frame, X_1 = R(z(X_0)) X_0 + t(X_0) with the frame's final grids (the
    recursion of Sec. 3.3), and the next frame starts from it."""
    from paper_2509_18097_gb300 import binding as B

    w = sphere_case(55)
    V = len(w.template)
    r = rng(56)
    tgt2 = synth.sinusoid(synth.sphere_points(r, 777), 0.12).astype(np.float32)
    ctx = B.pdg_create(B.pdg_config_default(res=w.res, payload="cayley"), w.template, w.edges, w.source,
                       max_pts=max(len(w.source), len(w.target), len(tgt2)))
    try:
        B.pdg_set_debug(ctx, True)
        B.pdg_begin_frame(ctx, w.target)
        for l, th in enumerate(w.thetas):
            B.pdg_write_theta(ctx, l, th.reshape(-1, 6))
        B.pdg_step(ctx, 3)
        th_end = [B.pdg_read(ctx, B.BUF_THETA, l, np.empty((n**3, 6), np.float32)) for l, n in enumerate(w.res)]
        B.pdg_end_frame(ctx)
        X1 = B.pdg_get_vertices(ctx, np.empty((V, 3), np.float32))
        ths = [t.reshape(n, n, n, 6).astype(np.float64) for t, n in zip(th_end, w.res)]
        H.check_close("X_1", X1, O.deform_cayley(w.template.astype(np.float64), ths, w.lo, w.hi))
        # pdg_deform applies the same transform to arbitrary points
        pts = synth.sphere_points(r, 333).astype(np.float32) * 1.1
        out = B.pdg_deform(ctx, pts, np.empty_like(pts))
        H.check_close("deform", out, O.deform_cayley(pts.astype(np.float64), ths, w.lo, w.hi))
        B.pdg_begin_frame(ctx, tgt2)
        th0 = [B.pdg_read(ctx, B.BUF_THETA, l, np.empty((n**3, 6), np.float32)) for l, n in enumerate(w.res)]
        assert all(not a.any() for a in th0)
        B.pdg_step(ctx, 1)
        w2 = synth.Workload("cayley_frame2", X1, w.edges, w.target, tgt2, w.res)
        g = dict(theta0=th0, **H.read_state(B, ctx, w2, C=6))
        B.pdg_end_frame(ctx)
    finally:
        B.pdg_destroy(ctx)
    H.stagewise(w2, g, H.oracle_cfg(w2, payload="cayley"))


def test_cayley_rejects_256_levels():
    from paper_2509_18097_gb300 import binding as B

    cfg = B.pdg_config_default(res=(16, 256), payload="cayley")
    assert B.pdg_query_bytes(cfg, 10, 10, 10) == 0
    v = np.zeros((3, 3), np.float32)
    with pytest.raises(B.PdgError) as e:
        B.pdg_create(cfg, v, np.zeros((0, 2), np.int32), v)
    assert e.value.status == B.ERR_INVALID


def test_cayley_batch_matches_solo_bitwise():
    """A Cayley job batched beside displacement jobs gives bitwise its solo results."""
    from paper_2509_18097_gb300 import binding as B

    jobs = [(sphere_case(57), "cayley"), (sphere_case(58, res=(2, 8)), "displacement"),
            (sphere_case(59, n_src=1500, res=(8, 16, 32)), "cayley")]

    def make(w, payload):
        ctx = B.pdg_create(B.pdg_config_default(res=w.res, payload=payload), w.template, w.edges, w.source,
                           max_pts=max(len(w.source), len(w.target)))
        B.pdg_begin_frame(ctx, w.target)
        return ctx

    def snap(ctx, w, payload):
        C = 6 if payload == "cayley" else 3
        out = {"loss": B.pdg_read(ctx, B.BUF_LOSS, 0, np.empty(4, np.float64)),
               "y": B.pdg_read(ctx, B.BUF_Y, 0, np.empty((len(w.template) + len(w.source), 3), np.float32))}
        for l, n in enumerate(w.res):
            out[l] = B.pdg_read(ctx, B.BUF_THETA, l, np.empty((n**3, C), np.float32))
        return out

    ref = []
    for w, pl in jobs:
        c = make(w, pl)
        B.pdg_step(c, 4)
        ref.append(snap(c, w, pl))
        B.pdg_destroy(c)
    ctxs = [make(w, pl) for w, pl in jobs]
    b = B.pdg_batch_create(4)
    try:
        B.pdg_batch_set(b, ctxs)
        B.pdg_batch_step(b, 4)
        for (w, pl), c, rf in zip(jobs, ctxs, ref):
            got = snap(c, w, pl)
            for k in rf:
                assert np.array_equal(got[k], rf[k]), (pl, k)
    finally:
        B.pdg_batch_destroy(b)
        for c in ctxs:
            B.pdg_destroy(c)
