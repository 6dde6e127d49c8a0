"""Shared machinery of the GPU parity tests: run steps through the C-ABI and compare with
the FP64 oracle.

Tolerance (from the arithmetic): every float comparison is
    |gpu - oracle| <= 1e-6 * S + 1e-5 * |oracle|
i.e. 1e-5 relative plus 1e-6 absolute in the units of the terms that make up the output.
S is max|oracle| for element-wise results, and for a sum the larger of that and the sum
of the absolute values of its terms (per element): FP32 rounds every term to ~6e-8 of
its own size, so a sum whose terms nearly cancel (the coarsest grid levels gather
hundreds of isometry terms of O(w_iso / |E|) that sum to ~0 by translation invariance) is
only determined to ~1e-7 of sum|terms|.  The preconditioner's six length-n FFT passes add
O(log2 n * 6e-8) of the level's norm.
Nearest-neighbour indices must match exactly except at near-ties (relative gap between
the best and second-best squared distance below 1e-6), which are counted and reported.
"""
from __future__ import annotations

import numpy as np

from oracle import pdg_oracle as O

RTOL = 1e-5
ATOL_REL = 1e-6
NEAR_TIE = 1e-6


def check_close(name, a, b, rtol=RTOL, atol_rel=ATOL_REL, mask=None, terms=None):
    """`terms`: per-element sum of the absolute values of the terms of each output (for
    sums), broadcastable to b."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    assert a.shape == b.shape, (name, a.shape, b.shape)
    S = np.full(b.shape, float(np.abs(b).max()) if b.size else 0.0)
    if terms is not None:
        S = np.maximum(S, np.broadcast_to(np.asarray(terms, np.float64), b.shape))
    if mask is not None:
        a, b, S = a[mask], b[mask], S[mask]
    if b.size == 0:
        return 0.0
    scale = float(S.max())
    err = np.abs(a - b)
    tol = atol_rel * S + rtol * np.abs(b)
    bad = err > tol
    worst = float((err / np.maximum(tol, 1e-300)).max())
    assert not bad.any(), (
        f"{name}: {int(bad.sum())} of {bad.size} entries outside |d| <= {atol_rel}*{scale:.3e} + {rtol}|ref|; "
        f"worst ratio {worst:.2f}"
    )
    return worst


def read_state(B, ctx, w, debug=True, C=3):
    """Every per-step buffer of a context after a step (host numpy arrays); C: payload channels."""
    V, N, M = len(w.template), len(w.source), len(w.target)
    out = {}
    out["y"] = B.pdg_read(ctx, B.BUF_Y, 0, np.empty((V + N, 3), np.float32))
    out["g_pts"] = B.pdg_read(ctx, B.BUF_POINT_GRAD, 0, np.empty((V + N, 3), np.float32))
    out["nn_fwd"] = B.pdg_read(ctx, B.BUF_NN_FWD, 0, np.empty(V + N, np.int32))
    out["nn_rev"] = B.pdg_read(ctx, B.BUF_NN_REV, 0, np.empty((2, M), np.int32))
    out["loss"] = B.pdg_read(ctx, B.BUF_LOSS, 0, np.empty(4, np.float64))
    out["counters"] = B.pdg_read(ctx, B.BUF_COUNTERS, 0, np.empty(4, np.uint64))
    out["grads"] = [B.pdg_read(ctx, B.BUF_GRAD, l, np.empty((n**3, C), np.float32)) for l, n in enumerate(w.res)]
    if debug:
        out["pgrads"] = [B.pdg_read(ctx, B.BUF_PGRAD, l, np.empty((n**3, C), np.float32)) for l, n in enumerate(w.res)]
    out["theta1"] = [B.pdg_read(ctx, B.BUF_THETA, l, np.empty((n**3, C), np.float32)) for l, n in enumerate(w.res)]
    return out


def is_close(a, b, rtol=RTOL, atol_rel=ATOL_REL):
    """check_close as a predicate (element-wise tolerance of an element-wise result)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    S = float(np.abs(b).max()) if b.size else 0.0
    return bool(np.all(np.abs(a - b) <= atol_rel * S + rtol * np.abs(b)))


def gpu_run(w, cfg_kwargs=None, thetas=None, steps=1, read=True, debug=True, count_nn=False):
    """Runs `steps` iterations of one frame through the C-ABI and reads every buffer."""
    import torch

    from paper_2509_18097_gb300 import binding as B

    cfg_kwargs = dict(cfg_kwargs or {})
    C = 6 if cfg_kwargs.get("payload") == "cayley" else 3
    cfg = B.pdg_config_default(res=w.res, lo=w.lo, hi=w.hi, **cfg_kwargs)
    mp = max(len(w.source), len(w.target))
    ctx = B.pdg_create(cfg, w.template, w.edges, w.source, max_pts=mp)
    try:
        if debug or count_nn:
            B.pdg_set_debug(ctx, debug, count_nn=count_nn)
        B.pdg_begin_frame(ctx, w.target)
        if thetas is not None:
            for l, th in enumerate(thetas):
                B.pdg_write_theta(ctx, l, np.asarray(th, np.float32).reshape(-1, C))
        th0 = [B.pdg_read(ctx, B.BUF_THETA, l, np.empty((n**3, C), np.float32)) for l, n in enumerate(w.res)]
        assert B.pdg_step_kernel_count(ctx) == 0  # no step graph before the first step
        B.pdg_step(ctx, steps)
        torch.cuda.synchronize()
        V, N, M = len(w.template), len(w.source), len(w.target)
        out = dict(theta0=th0, kernels_per_step=B.pdg_step_kernel_count(ctx))
        if read:
            out.update(read_state(B, ctx, w, debug, C))
        st = B.pdg_end_frame(ctx)
        out["stats"] = st
        out["verts"] = B.pdg_get_vertices(ctx, np.empty((V, 3), np.float32))
        return out
    finally:
        B.pdg_destroy(ctx)


def oracle_cfg(w, **kw):
    return O.Config(res=tuple(w.res), lo=tuple(w.lo), hi=tuple(w.hi), **kw)


def nn_check(name, gpu_idx, q, b):
    """Exact NN of fp32 queries q in b (oracle) vs the GPU indices; returns the number of
    near-ties and the mask of queries whose index differs."""
    idx, d2 = O.nn_exact(q, b)
    gap = O.nn_second_gap(q, b, idx, d2)
    near = gap < NEAR_TIE
    diff = idx != gpu_idx
    assert not (diff & ~near).any(), f"{name}: {int((diff & ~near).sum())} index mismatches away from near-ties"
    return int(near.sum()), diff


def stagewise(w, g, cfg: O.Config, check_adam=True):
    """Checks every stage of one GPU step against the oracle applied to the GPU's own
    input of that stage.  Returns a dict of counts for reporting."""
    V, N, M = len(w.template), len(w.source), len(w.target)
    C = cfg.channels
    x = np.concatenate([w.template, w.source]).astype(np.float64)
    th0 = [t.reshape(n, n, n, C).astype(np.float64) for t, n in zip(g["theta0"], w.res)]
    # (a) evaluation (the Cayley payload: y = R(z(x)) x + t(x))
    deform = O.deform_cayley if cfg.payload == "cayley" else O.deform
    check_close("y", g["y"], deform(x, th0, cfg.lo, cfg.hi))
    y = g["y"].astype(np.float64)
    P = w.target.astype(np.float64)
    # (b) nearest neighbours, all four directions
    t1, d1 = nn_check("nn X->P", g["nn_fwd"][:V], y[:V], P)
    t2, d2 = nn_check("nn Phat->P", g["nn_fwd"][V:], y[V:], P)
    t3, d3 = nn_check("nn P->X", g["nn_rev"][0], P, y[:V])
    t4, d4 = nn_check("nn P->Phat", g["nn_rev"][1], P, y[V:])
    # losses and point gradients on the GPU's deformed points
    cm = O.robust_chamfer(y[:V], P, cfg.alpha, cfg.robust_weight_stopgrad)
    cp = O.robust_chamfer(y[V:], P, cfg.alpha, cfg.robust_weight_stopgrad)
    e_prev = O.edge_lengths(w.template.astype(np.float64), w.edges)
    iso, giso = O.isometry(y[:V], w.edges, e_prev)
    loss = cfg.w_chamfer_mesh * cm["loss"] + cfg.w_chamfer_pts * cp["loss"] + cfg.w_iso * iso
    ties = t1 + t2 + t3 + t4
    # the robust Chamfer loss is continuous at a nearest-neighbour tie (both candidates have
    # the same squared distance), so the losses are compared whatever the tie count
    check_close("loss", g["loss"], [loss, cm["loss"], cp["loss"], iso])
    gref = np.concatenate([cfg.w_chamfer_mesh * cm["grad_A"] + cfg.w_iso * giso, cfg.w_chamfer_pts * cp["grad_A"]])
    # points whose gradient involves a near-tie assignment or a near-kink edge are excluded
    excl = np.zeros(V + N, bool)
    excl[:V] |= d1
    excl[V:] |= d2
    for dmask, off, own in ((d3, 0, g["nn_rev"][0]), (d4, V, g["nn_rev"][1])):
        excl[off + own[dmask]] = True
        excl[off + (cm if off == 0 else cp)["nn_ba"][dmask]] = True
    r = O.edge_lengths(y[:V], w.edges) - e_prev
    kink = (r != 0) & (np.abs(r) < 1e-6 * np.maximum(e_prev, 1e-12))
    excl[np.asarray(w.edges)[kink].ravel()] = True
    check_close("point grads", g["g_pts"], gref, mask=~excl)
    # (d) adjoint of the GPU's point gradients (through the transform's backward with the
    # Cayley payload)
    gp = g["g_pts"].astype(np.float64)
    if cfg.payload == "cayley":
        gp = O.apply_transform_backward(x, O.eval_displacement(x, th0, cfg.lo, cfg.hi), gp)
    adj = O.interp_adjoint(x, gp, cfg.res, cfg.lo, cfg.hi)
    adj_abs = O.interp_adjoint(x, np.abs(gp), cfg.res, cfg.lo, cfg.hi)  # sum of |terms| per vertex
    for l, n in enumerate(cfg.res):
        check_close(f"grad level {l}", g["grads"][l], adj[l].reshape(-1, C), terms=adj_abs[l].reshape(-1, C))
    # (e) preconditioner on the GPU's grid gradients, then Adam on the GPU's result; levels
    # above 64^3 use the oracle's eigen-decomposition form of the same operator (CG on them
    # takes minutes)
    for l, n in enumerate(cfg.res):
        gl = g["grads"][l].reshape(n, n, n, C).astype(np.float64)
        if not cfg.precondition:
            pg = gl
        elif n > 64:
            pg = O.sobolev_precondition_spectral(gl, cfg.lam(l))
        else:
            pg = O.sobolev_precondition(gl, cfg.lam(l))
        if "pgrads" in g:
            check_close(f"pgrad level {l}", g["pgrads"][l], pg.reshape(-1, C))
        if check_adam:
            src = g["pgrads"][l].astype(np.float64) if "pgrads" in g else pg.reshape(-1, C)
            t1_, _, _ = O.adam_update(th0[l].reshape(-1, C), 0.0, 0.0, src, 1, cfg.lr(l), cfg.beta1, cfg.beta2, cfg.eps)
            check_close(f"theta level {l}", g["theta1"][l], t1_)
    return dict(near_ties=ties, near_kinks=int(kink.sum()), excluded_points=int(excl.sum()))
