"""torch.autograd.Function over the hand-written backward kernels (trilinear adjoint,
robust-Chamfer gradient, isometry gradient) at the headline size (50 412 vertices,
100k + 100k points, 16^3..128^3, grids N(0, 0.01^2)):

* against FP64 central finite differences (h = 1e-4) on 1000 random grid entries, and
* against the oracle's reference gradient.

A central difference is evaluated exactly and locally: perturbing entry (l, v, c) moves
only the points whose level-l cell has v as a corner, so with every nearest-neighbour
assignment and isometry sign unchanged inside the stencil, L(+h) - L(-h) is the change of
the forward terms of those points, of the reverse terms of the targets matched to them and
of their incident edges.  Entries whose stencil changes an assignment or a sign (a kink of
the piecewise-smooth loss) are excluded and counted; the local evaluator itself is checked
against the full oracle loss on a small problem (`test_local_difference_equals_full_loss`).
"""
import numpy as np
import pytest

from oracle import pdg_oracle as O
from paper_2509_18097_gb300 import synth
from tests import gpu_helpers as H


class LocalFD:
    """Exact FP64 loss differences for single grid-entry perturbations."""

    def __init__(self, w, cfg, thetas):
        from scipy.spatial import cKDTree

        self.cfg = cfg
        self.V = len(w.template)
        self.x = np.concatenate([w.template, w.source]).astype(np.float64)
        self.th = [np.asarray(t, np.float64) for t in thetas]
        self.y = O.deform(self.x, self.th, cfg.lo, cfg.hi)
        self.P = w.target.astype(np.float64)
        self.E = np.asarray(w.edges, np.int64)
        self.e_prev = O.edge_lengths(w.template.astype(np.float64), self.E)
        V = self.V
        self.sets = [(0, V), (V, len(self.x))]
        self.tP = cKDTree(self.P)
        self.fwd_idx, self.fwd_d2 = O.nn_exact(self.y, self.P)
        self.rev = []
        for lo, hi in self.sets:
            idx, d2 = O.nn_exact(self.P, self.y[lo:hi])
            self.rev.append((idx + lo, d2, cKDTree(self.y[lo:hi])))
        self.inc = [[] for _ in range(V)]
        for e, (i, j) in enumerate(self.E):
            self.inc[i].append(e)
            self.inc[j].append(e)
        self.corners = [O._corners(self.x, cfg.lo, cfg.hi, n) for n in cfg.res]

    def phi(self, s):
        return s * np.exp(-self.cfg.alpha * s)

    def weight(self, p):
        c = self.cfg
        return c.w_chamfer_mesh if p < self.V else c.w_chamfer_pts

    def delta(self, l, v, ch, h):
        """(L(theta + h e) - L(theta - h e), ok); ok False if an assignment or sign changes."""
        cfg = self.cfg
        idx, w = self.corners[l]
        hit = np.nonzero(idx == v)
        S = hit[0]
        if len(S) == 0:
            return 0.0, True
        wS = w[hit] / len(cfg.res)
        out = []
        for sgn in (1.0, -1.0):
            ynew = self.y[S].copy()
            ynew[:, ch] += sgn * h * wS
            dL = 0.0
            # forward terms of the moved points (same nearest target required)
            ni, nd = O.nn_exact(ynew, self.P)
            if not np.array_equal(ni, self.fwd_idx[S]):
                return 0.0, False
            for k, p in enumerate(S):
                nA = self.V if p < self.V else len(self.x) - self.V
                dL += self.weight(p) / nA * (self.phi(nd[k]) - self.phi(self.fwd_d2[p]))
            # reverse terms: targets matched to moved points keep them, no target gets a
            # moved point closer than its match
            for si, (lo, hi) in enumerate(self.sets):
                Sset = S[(S >= lo) & (S < hi)]
                if len(Sset) == 0:
                    continue
                ridx, rd2, tree = self.rev[si]
                ynew_set = ynew[(S >= lo) & (S < hi)]
                rmax = np.sqrt(rd2.max()) + 2 * h
                cand = set()
                for q in ynew_set:
                    cand.update(self.tP.query_ball_point(q, rmax))
                cand.update(np.nonzero(np.isin(ridx, Sset))[0].tolist())
                wset = self.weight(lo)
                M = len(self.P)
                for t in cand:
                    tp = self.P[t]
                    d_new = ((ynew_set - tp) ** 2).sum(1)
                    owner = ridx[t]
                    if owner in Sset:
                        k = int(np.nonzero(Sset == owner)[0][0])
                        s_new = d_new[k]
                        others = np.delete(d_new, k)
                        others_idx = np.delete(Sset, k)
                        kk = min(len(Sset) + 2, hi - lo)
                        dd, ii = tree.query(tp, k=kk)
                        ii = np.atleast_1d(ii) + lo
                        nonS = [(((self.y[j] - tp) ** 2).sum(), j) for j in ii if j not in Sset]
                        best_other = min(nonS) if nonS else (np.inf, -1)
                        comp = [(s_new, owner)] + list(zip(others, others_idx)) + [best_other]
                        if min(comp) != (s_new, owner):
                            return 0.0, False
                        dL += wset / M * (self.phi(s_new) - self.phi(rd2[t]))
                    else:
                        cur = (rd2[t], owner)
                        if any((d, j) < cur for d, j in zip(d_new, Sset)):
                            return 0.0, False
            # isometry over edges incident to moved template vertices (same signs)
            if cfg.w_iso:
                ymod = {int(p): ynew[k] for k, p in enumerate(S) if p < self.V}
                edges = set()
                for p in ymod:
                    edges.update(self.inc[p])
                for e in edges:
                    i, j = self.E[e]
                    yi = ymod.get(int(i), self.y[i])
                    yj = ymod.get(int(j), self.y[j])
                    r_old = np.linalg.norm(self.y[i] - self.y[j]) - self.e_prev[e]
                    r_new = np.linalg.norm(yi - yj) - self.e_prev[e]
                    if np.sign(r_old) != np.sign(r_new) or r_old == 0:
                        return 0.0, False
                    dL += cfg.w_iso / len(self.E) * (abs(r_new) - abs(r_old))
            out.append(dL)
        return out[0] - out[1], True


def test_local_difference_equals_full_loss():
    """Pin of the local evaluator: on a small problem it equals the difference of two full
    oracle losses."""
    r = np.random.Generator(np.random.PCG64(3))
    v, _, e = synth.icosphere(1)
    src = synth.sphere_points(r, 120).astype(np.float32)
    tgt = synth.sinusoid(synth.sphere_points(r, 150), 0.1).astype(np.float32)
    w = synth.Workload("fd_small", v, e, src, tgt, (3, 5))
    cfg = H.oracle_cfg(w)
    th = [r.standard_normal((n, n, n, 3)) * 0.02 for n in w.res]
    fd = LocalFD(w, cfg, th)
    h = 1e-4
    checked = 0
    for l, n in enumerate(w.res):
        for v_ in range(n**3):
            for ch in range(3):
                d, ok = fd.delta(l, v_, ch, h)
                if not ok:
                    continue
                tp = [t.copy() for t in th]
                tm = [t.copy() for t in th]
                tp[l].reshape(-1, 3)[v_, ch] += h
                tm[l].reshape(-1, 3)[v_, ch] -= h
                Lp = O.step(O.begin_frame(w.template, w.source, w.target, w.edges, cfg, tp), cfg, update=False)["loss"]
                Lm = O.step(O.begin_frame(w.template, w.source, w.target, w.edges, cfg, tm), cfg, update=False)["loss"]
                assert abs(d - (Lp - Lm)) <= 1e-12 + 1e-9 * abs(Lp - Lm), (l, v_, ch, d, Lp - Lm)
                checked += 1
    assert checked > 100


@pytest.mark.gpu
def test_grid_loss_function_vs_finite_differences_and_oracle():
    import torch

    from paper_2509_18097_gb300 import binding as B
    from paper_2509_18097_gb300.autograd import grid_loss

    w = synth.ellipsoid_pair(seed=0)
    cfg = H.oracle_cfg(w)
    dev = torch.device("cuda")
    ctx = B.pdg_create(B.pdg_config_default(res=w.res), w.template, w.edges, w.source, max_pts=len(w.target))
    try:
        B.pdg_begin_frame(ctx, w.target)
        thetas = [torch.tensor(t, device=dev, requires_grad=True) for t in w.thetas]
        loss = grid_loss(ctx, thetas)
        loss.backward()
        grads = [t.grad.detach().cpu().numpy().reshape(-1, 3).astype(np.float64) for t in thetas]
        B.pdg_end_frame(ctx)
    finally:
        B.pdg_destroy(ctx)
    th64 = [t.astype(np.float64) for t in w.thetas]
    # oracle reference gradient (FP64) at the same grids
    st = O.begin_frame(w.template, w.source, w.target, w.edges, cfg, th64)
    o = O.step(st, cfg, update=False)
    assert abs(float(loss) - o["loss"]) <= 1e-5 * abs(o["loss"])
    x = st.x
    gabs = O.interp_adjoint(x, np.abs(o["g_pts"]), cfg.res, cfg.lo, cfg.hi)
    # vertices whose support holds a point with a near-tie match are excluded from the
    # oracle comparison (their gradient depends on which of two equidistant points wins)
    V = len(w.template)
    y = o["y"]
    near = np.zeros(len(x), bool)
    for (q, b, gi) in ((y[:V], w.target, slice(0, V)), (y[V:], w.target, slice(V, None))):
        idx, d2 = O.nn_exact(q, b.astype(np.float64))
        near[gi] |= O.nn_second_gap(q, b.astype(np.float64), idx, d2) < H.NEAR_TIE
    sus = O.interp_adjoint(x, np.repeat(near[:, None].astype(float), 3, 1), cfg.res, cfg.lo, cfg.hi)
    for l in range(len(w.res)):
        mask = sus[l].reshape(-1, 3)[:, 0] == 0
        H.check_close(f"autograd vs oracle level {l}", grads[l][mask], o["grads"][l].reshape(-1, 3)[mask],
                      terms=gabs[l].reshape(-1, 3)[mask])
    # central differences on 1000 random entries (half of them where the gradient is nonzero)
    fd = LocalFD(w, cfg, th64)
    r = np.random.Generator(np.random.PCG64(7))
    picks = []
    for _ in range(500):
        l = int(r.integers(len(w.res)))
        nz = np.nonzero(np.abs(grads[l]).sum(1))[0]
        picks.append((l, int(r.choice(nz)), int(r.integers(3))))
        l2 = int(r.integers(len(w.res)))
        picks.append((l2, int(r.integers(w.res[l2] ** 3)), int(r.integers(3))))
    h = 1e-4
    excluded = 0
    for l, v_, ch in picks:
        d, ok = fd.delta(l, v_, ch, h)
        if not ok:
            excluded += 1
            continue
        g_fd = d / (2 * h)
        g = grads[l][v_, ch]
        S = gabs[l].reshape(-1, 3)[v_, ch]
        assert abs(g - g_fd) <= 1e-5 * abs(g_fd) + 1e-6 * max(S, np.abs(grads[l]).max()), (l, v_, ch, g, g_fd)
    print(f"finite differences: {len(picks) - excluded} entries checked, {excluded} excluded (assignment/sign change)")
    assert excluded < 100
