"""Batching, serving, checkpointing and API behaviour on the GPU (through the C-ABI).

The step is deterministic (no floating-point atomics), so a context's results must be
bitwise identical alone, inside any batch, across membership changes, through the server
and after a save/load round trip."""
import numpy as np
import pytest

from oracle import pdg_oracle as O
from paper_2509_18097_gb300 import synth
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def rng(s):
    return np.random.Generator(np.random.PCG64(s))


def job(seed, sub=2, n_src=600, n_tgt=750, res=(4, 8, 16)):
    r = rng(seed)
    v, _, e = synth.icosphere(sub)
    src = synth.sphere_points(r, n_src).astype(np.float32)
    tgt = synth.sinusoid(synth.sphere_points(r, n_tgt), 0.1).astype(np.float32)
    return synth.Workload(f"job{seed}", v, e, src, tgt, res)


JOBS = [job(0), job(1, sub=1, n_src=300, n_tgt=1300, res=(2, 8)), job(2, sub=3, n_src=2000, n_tgt=900, res=(8, 16, 32, 64))]


def make(B, w):
    ctx = B.pdg_create(B.pdg_config_default(res=w.res), w.template, w.edges, w.source,
                       max_pts=max(len(w.source), len(w.target)))
    B.pdg_begin_frame(ctx, w.target)
    return ctx


def snapshot(B, ctx, w):
    out = {"loss": B.pdg_read(ctx, B.BUF_LOSS, 0, np.empty(4, np.float64)),
           "y": B.pdg_read(ctx, B.BUF_Y, 0, np.empty((len(w.template) + len(w.source), 3), np.float32))}
    for l, n in enumerate(w.res):
        out[f"theta{l}"] = B.pdg_read(ctx, B.BUF_THETA, l, np.empty((n**3, 3), np.float32))
    return out


def solo(B, w, steps):
    ctx = make(B, w)
    B.pdg_step(ctx, steps)
    s = snapshot(B, ctx, w)
    B.pdg_destroy(ctx)
    return s


def test_batch_matches_solo_bitwise():
    from paper_2509_18097_gb300 import binding as B

    steps = 4
    ref = [solo(B, w, steps) for w in JOBS]
    ctxs = [make(B, w) for w in JOBS]
    b = B.pdg_batch_create(8)
    B.pdg_batch_set(b, ctxs)
    B.pdg_batch_step(b, steps)
    for w, c, r in zip(JOBS, ctxs, ref):
        s = snapshot(B, c, w)
        for k in r:
            assert np.array_equal(s[k], r[k]), (w.name, k)
        B.pdg_destroy(c)
    B.pdg_batch_destroy(b)


def test_batch_membership_changes():
    """Jobs join and leave between iterations; each still matches its solo run."""
    from paper_2509_18097_gb300 import binding as B

    ref = [solo(B, w, 5) for w in JOBS]
    ctxs = [make(B, w) for w in JOBS]
    b = B.pdg_batch_create(4)
    B.pdg_batch_set(b, ctxs[:1])
    B.pdg_batch_step(b, 2)               # job 0: 2
    B.pdg_batch_set(b, ctxs[:2])
    B.pdg_batch_step(b, 1)               # job 0: 3, job 1: 1
    B.pdg_batch_set(b, [ctxs[2], ctxs[1]])
    B.pdg_batch_step(b, 4)               # job 1: 5, job 2: 4
    B.pdg_step(ctxs[0], 2)               # job 0: 5 alone
    B.pdg_batch_set(b, [ctxs[2]])
    B.pdg_batch_step(b, 1)               # job 2: 5
    for w, c, r in zip(JOBS, ctxs, ref):
        s = snapshot(B, c, w)
        for k in r:
            assert np.array_equal(s[k], r[k]), (w.name, k)
        B.pdg_destroy(c)
    B.pdg_batch_destroy(b)


def seq_set(n_seq=4, n_frames=3):
    seqs = []
    for i in range(n_seq):
        r = rng(100 + i)
        v, _, e = synth.icosphere(1 + i % 2)
        base = synth.sphere_points(r, 500 + 97 * i)
        frames = [synth.sinusoid(base, 0.03 * (k + 1)).astype(np.float32) for k in range(n_frames)]
        from paper_2509_18097_gb300.serve import Sequence

        seqs.append(Sequence(i, v, e, base.astype(np.float32), frames, (4, 8, 16)[: 2 + i % 2], 600 + 97 * 4))
    return seqs


@pytest.mark.parametrize("order", ["fifo", "size"])
def test_server_results_equal_plain_and_solo(order):
    """Whatever the admission order, every frame's result is bitwise the one the plain
    one-at-a-time form gives."""
    from paper_2509_18097_gb300 import serve

    seqs = seq_set()
    trace_a = serve.poisson_trace(seqs, rate_hz=2000.0, seed=1)
    trace_b = serve.poisson_trace(seqs, rate_hz=2000.0, seed=1)
    srv = serve.Server(seqs, steps=6, budget_bytes=8 * 1024**3, max_slots=3, order=order)
    stats = srv.run(trace_a, realtime=False)
    srv.close()
    plain = serve.serve_plain(seqs, trace_b, steps=6, realtime=False)
    assert stats["frames"] == plain["frames"] == sum(len(s.frames) for s in seqs)
    last_a = {r.sid: r for r in trace_a if r.vertices is not None}
    last_b = {r.sid: r for r in trace_b if r.vertices is not None}
    for sid in last_a:
        assert np.array_equal(last_a[sid].vertices, last_b[sid].vertices), sid
    la = sorted((r.sid, r.frame, r.loss) for r in trace_a)
    lb = sorted((r.sid, r.frame, r.loss) for r in trace_b)
    assert la == lb


def test_server_respects_memory_budget():
    from paper_2509_18097_gb300 import binding as B
    from paper_2509_18097_gb300 import serve

    seqs = seq_set(n_seq=3, n_frames=2)
    need = max(B.pdg_query_bytes(B.pdg_config_default(res=s.res), len(s.template), len(s.edges), s.max_pts)
               for s in seqs)
    srv = serve.Server(seqs, steps=3, budget_bytes=int(need * 1.5), max_slots=8)
    peak = [0]
    orig = srv._open

    def watch(s):
        ok = orig(s)
        peak[0] = max(peak[0], srv.used)
        return ok

    srv._open = watch
    stats = srv.run(serve.poisson_trace(seqs, 5000.0, seed=2), realtime=False)
    srv.close()
    assert stats["frames"] == 6
    assert peak[0] <= int(need * 1.5)


def test_save_load_state_continues_bitwise():
    from paper_2509_18097_gb300 import binding as B

    w = JOBS[0]
    f2 = synth.sinusoid(w.target, 0.02).astype(np.float32)
    a = make(B, w)
    B.pdg_step(a, 3)
    B.pdg_end_frame(a)
    blob = B.pdg_save_state(a)
    B.pdg_fit_frame(a, f2, 3)
    va = B.pdg_get_vertices(a, np.empty((len(w.template), 3), np.float32))
    c = B.pdg_create(B.pdg_config_default(res=w.res), w.template, w.edges, w.source,
                     max_pts=max(len(w.source), len(w.target)))
    B.pdg_load_state(c, blob)
    B.pdg_fit_frame(c, f2, 3)
    vc = B.pdg_get_vertices(c, np.empty((len(w.template), 3), np.float32))
    assert np.array_equal(va, vc)
    B.pdg_destroy(a)
    B.pdg_destroy(c)


def test_host_and_device_buffers_agree():
    import torch

    from paper_2509_18097_gb300 import binding as B

    w = JOBS[1]
    dev = torch.device("cuda")
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    cfg = B.pdg_config_default(res=w.res)
    a = B.pdg_create(cfg, w.template, w.edges, w.source, max_pts=2000)
    b = B.pdg_create(cfg, T(w.template), T(w.edges), T(w.source), max_pts=2000)
    sa = B.pdg_fit_frame(a, w.target, 4)
    sb = B.pdg_fit_frame(b, T(w.target), 4)
    assert sa.loss_total == sb.loss_total
    va = B.pdg_get_vertices(a, np.empty((len(w.template), 3), np.float32))
    vb = B.pdg_get_vertices(b, torch.empty((len(w.template), 3), device=dev)).cpu().numpy()
    assert np.array_equal(va, vb)
    B.pdg_destroy(a)
    B.pdg_destroy(b)


def test_deform_matches_oracle():
    from paper_2509_18097_gb300 import binding as B

    w = JOBS[2]
    ctx = make(B, w)
    B.pdg_step(ctx, 3)
    th = [B.pdg_read(ctx, B.BUF_THETA, l, np.empty((n**3, 3), np.float32)).reshape(n, n, n, 3).astype(np.float64)
          for l, n in enumerate(w.res)]
    p = rng(5).uniform(-1.7, 1.7, (5003, 3)).astype(np.float32)
    out = B.pdg_deform(ctx, p, np.empty_like(p))
    H.check_close("deform", out, O.deform(p.astype(np.float64), th, (-1.5,) * 3, (1.5,) * 3))
    B.pdg_destroy(ctx)


def test_errors_are_statuses_not_faults():
    from paper_2509_18097_gb300 import binding as B

    w = JOBS[0]
    ctx = B.pdg_create(B.pdg_config_default(res=w.res), w.template, w.edges, w.source, max_pts=1000)
    with pytest.raises(B.PdgError) as e:
        B.pdg_step(ctx, 1)  # outside a frame
    assert e.value.status == B.ERR_STATE
    bad = w.target.copy()
    bad[7, 1] = np.nan
    with pytest.raises(B.PdgError) as e:
        B.pdg_begin_frame(ctx, bad)
    assert e.value.status == B.ERR_INVALID
    with pytest.raises(B.PdgError) as e:
        B.pdg_begin_frame(ctx, np.zeros((1001, 3), np.float32))  # above max_pts
    assert e.value.status == B.ERR_BUDGET
    B.pdg_begin_frame(ctx, w.target)
    with pytest.raises(B.PdgError) as e:
        B.pdg_begin_frame(ctx, w.target)  # already open
    assert e.value.status == B.ERR_STATE
    B.pdg_step(ctx, 1)
    B.pdg_end_frame(ctx)
    B.pdg_destroy(ctx)
