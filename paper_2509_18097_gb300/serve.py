"""Continuous-batching server of per-frame fitting requests.

Requests are frames of independent point-cloud sequences (Sec. 3: each frame fits the
grid G_t that maps frame t-1 to frame t).  Frames of one sequence are served in order;
frames of different sequences overlap on the device:

* every sequence owns one resident context (template, current source cloud, grids and
  optimiser state stay on the device across frames), created on its first request if the
  device-memory budget allows (`pdg_query_bytes`), otherwise the request waits;
* at every boundary of at most `chunk` iterations the server admits waiting frames whose
  sequence is idle (`pdg_begin_frame`, on a side stream, from host memory), retires finished
  frames (`pdg_end_frame`), and runs the next iterations of every live frame, each one CUDA-
  graph launch of batched kernels (`pdg_batch_step`);
* the batch has `max_slots` slots; a sequence's context is released when its last frame
  is done, freeing budget for new sequences.

`serve_plain` runs the same trace one frame at a time (`pdg_fit_frame`), the baseline the
batched form is compared with.  Latency = finish time - arrival time of each frame.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np


@dataclasses.dataclass
class Sequence:
    """One sequence of the trace: template mesh, first cloud, frames and grid config."""

    sid: int
    template: np.ndarray
    edges: np.ndarray
    source0: np.ndarray
    frames: list  # [n_frames] float32 [M, 3]
    res: tuple
    max_pts: int


@dataclasses.dataclass
class Request:
    sid: int
    frame: int
    arrival: float  # seconds from the trace start
    admitted: float = -1.0
    finished: float = -1.0
    loss: float = float("nan")
    vertices: np.ndarray | None = None


def poisson_trace(seqs, rate_hz: float, seed: int = 0):
    """Requests of all frames of all sequences with Poisson arrivals at `rate_hz`; frame k
    of a sequence never arrives before frame k-1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pending = {s.sid: 0 for s in seqs}
    order = []
    total = sum(len(s.frames) for s in seqs)
    t = 0.0
    sids = [s.sid for s in seqs]
    while len(order) < total:
        t += rng.exponential(1.0 / rate_hz)
        live = [sid for sid in sids if pending[sid] < len(next(s for s in seqs if s.sid == sid).frames)]
        sid = live[rng.integers(len(live))]
        order.append(Request(sid, pending[sid], t))
        pending[sid] += 1
    return order


def frame_cost(s: Sequence, frame: int) -> float:
    """Estimated device bytes of one iteration of a frame: about 200 B per query and target
    point (evaluation, searches, gradients) and 100 B per grid vertex (adjoint, preconditioner,
    Adam).  Used only to order admissions."""
    return 200.0 * (len(s.template) + len(s.source0) + 2 * len(s.frames[frame])) + 100.0 * sum(n**3 for n in s.res)


def _percentiles(lat):
    lat = np.asarray(lat)
    return float(np.percentile(lat, 50)), float(np.percentile(lat, 99))


class Server:
    """Continuous batching of per-frame fitting requests on one GPU.

    `chunk` bounds the iterations one batch launch runs, so a frame that arrives while
    others are on the GPU joins them at the next boundary of at most `chunk` iterations
    (its set-up runs on a side stream meanwhile, from host memory); the host stays at most one
    chunk ahead of the GPU.  `order` picks which waiting frames fill free slots: "fifo" in
    arrival order, "size" the smallest estimated work first (frame_cost); either way only
    the next frame of each sequence is eligible, so a sequence's frames stay in order."""

    def __init__(self, seqs, steps: int, budget_bytes: int, max_slots: int = 64, device=None, cfg_kwargs=None,
                 chunk: int = 4, order: str = "fifo"):
        import torch

        from . import binding as B

        self.B = B
        self.torch = torch
        self.dev = device or torch.device("cuda")
        self.seqs = {s.sid: s for s in seqs}
        self.steps = steps
        self.budget = budget_bytes
        self.max_slots = max_slots
        self.chunk = max(1, int(chunk))
        if order not in ("fifo", "size"):
            raise ValueError("order must be 'fifo' or 'size'")
        self.order = order
        self.cfg_kwargs = cfg_kwargs or {}
        self.used = 0
        self.ctx = {}  # sid -> context handle
        self.bytes = {}
        self.batch = B.pdg_batch_create(max_slots)
        # two non-blocking streams (neither waits for the legacy default stream): batched
        # iterations on `main`, frame set-up on `admit`
        self.main = torch.cuda.Stream(self.dev)
        self.admit = torch.cuda.Stream(self.dev)

    def _cfg(self, s):
        return self.B.pdg_config_default(res=s.res, **self.cfg_kwargs)

    def _open(self, s):
        need = self.B.pdg_query_bytes(self._cfg(s), len(s.template), len(s.edges), s.max_pts)
        if self.used + need > self.budget:
            return False
        # host arrays: the library copies them on the side stream
        self.ctx[s.sid] = self.B.pdg_create(self._cfg(s), s.template, s.edges, s.source0, max_pts=s.max_pts,
                                            stream=self.admit.cuda_stream)
        self.bytes[s.sid] = need
        self.used += need
        return True

    def _close(self, sid):
        self.B.pdg_destroy(self.ctx.pop(sid))
        self.used -= self.bytes.pop(sid)

    def run(self, trace, realtime: bool = True):
        """Serves the trace; returns per-request records and summary statistics."""
        B = self.B
        main = self.main.cuda_stream
        waiting = collections.deque(sorted(trace, key=lambda r: r.arrival))
        arrived: list[Request] = []
        live = {}  # sid -> [request, steps done]
        busy = set()
        remaining = {sid: len(s.frames) for sid, s in self.seqs.items()}
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        members_changed = True
        prev_ev = None
        while waiting or arrived or live:
            t = now()
            while waiting and (waiting[0].arrival <= t or not realtime):
                arrived.append(waiting.popleft())
            # admit frames in arrival order: sequence idle, slot free, context resident; their
            # set-up runs on the side stream (host target copied by the library), beside the
            # batch's iterations on the main stream
            admitted = False
            # the next frame of each idle sequence, in the admission order
            firsts = {}
            for r in arrived:
                if r.sid not in busy and (r.sid not in firsts or r.frame < firsts[r.sid].frame):
                    firsts[r.sid] = r
            cand = sorted(firsts.values(), key=lambda r: (frame_cost(self.seqs[r.sid], r.frame), r.arrival)
                          if self.order == "size" else (r.arrival,))
            for r in cand:
                if len(live) >= self.max_slots:
                    break
                if r.sid in busy:
                    continue
                s = self.seqs[r.sid]
                if r.sid not in self.ctx and not self._open(s):
                    continue
                B.pdg_begin_frame(self.ctx[r.sid], s.frames[r.frame], stream=self.admit.cuda_stream)
                r.admitted = now()
                live[r.sid] = [r, 0]
                busy.add(r.sid)
                arrived.remove(r)
                members_changed = True
                admitted = True
            if admitted:
                self.main.wait_stream(self.admit)  # new members' set-up precedes their first step
            if not live:
                if waiting and realtime:
                    time.sleep(max(0.0, min(waiting[0].arrival - now(), 0.001)))
                continue
            if members_changed:
                B.pdg_batch_set(self.batch, [self.ctx[sid] for sid in live])
                members_changed = False
            # at most `chunk` iterations, fewer if a frame finishes sooner
            k = min(self.chunk, min(self.steps - st for _, st in live.values()))
            B.pdg_batch_step(self.batch, k, stream=main)
            ev = self.torch.cuda.Event()
            ev.record(self.main)
            finished = False
            for sid in list(live):
                live[sid][1] += k
                r, st = live[sid]
                if st >= self.steps:
                    stats = B.pdg_end_frame(self.ctx[sid], stream=main)  # synchronises the main stream
                    r.finished = now()
                    r.loss = stats.loss_total
                    del live[sid]
                    busy.discard(sid)
                    remaining[sid] -= 1
                    members_changed = True
                    finished = True
                    if remaining[sid] == 0:
                        r.vertices = B.pdg_get_vertices(self.ctx[sid], np.empty((len(self.seqs[sid].template), 3),
                                                                                np.float32), stream=main)
                        self._close(sid)
            if not finished and prev_ev is not None:
                prev_ev.synchronize()  # at most one chunk queued ahead of the GPU
            prev_ev = ev
        wall = now()
        lat = [r.finished - r.arrival for r in trace]
        p50, p99 = _percentiles(lat)
        return dict(frames=len(trace), wall_s=wall, frames_per_s=len(trace) / wall, p50_s=p50, p99_s=p99)

    def close(self):
        for sid in list(self.ctx):
            self._close(sid)
        self.B.pdg_batch_destroy(self.batch)


def serve_plain(seqs, trace, steps: int, device=None, cfg_kwargs=None, realtime: bool = True):
    """One frame at a time in arrival order (pdg_fit_frame), contexts resident per sequence."""
    import torch

    from . import binding as B

    dev = device or torch.device("cuda")
    byid = {s.sid: s for s in seqs}
    ctx = {}
    remaining = {s.sid: len(s.frames) for s in seqs}
    stream = torch.cuda.current_stream(dev).cuda_stream
    t0 = time.perf_counter()
    now = lambda: time.perf_counter() - t0
    for r in sorted(trace, key=lambda r: r.arrival):
        if realtime and r.arrival > now():
            time.sleep(r.arrival - now())
        s = byid[r.sid]
        if r.sid not in ctx:  # host arrays: the library copies them
            ctx[r.sid] = B.pdg_create(B.pdg_config_default(res=s.res, **(cfg_kwargs or {})), s.template,
                                      s.edges, s.source0, max_pts=s.max_pts, stream=stream)
        r.admitted = now()
        st = B.pdg_fit_frame(ctx[r.sid], s.frames[r.frame], steps, stream=stream)
        r.finished = now()
        r.loss = st.loss_total
        remaining[r.sid] -= 1
        if remaining[r.sid] == 0:
            r.vertices = B.pdg_get_vertices(ctx[r.sid], np.empty((len(s.template), 3), np.float32), stream=stream)
            B.pdg_destroy(ctx.pop(r.sid))
    wall = now()
    lat = [r.finished - r.arrival for r in trace]
    p50, p99 = _percentiles(lat)
    return dict(frames=len(trace), wall_s=wall, frames_per_s=len(trace) / wall, p50_s=p50, p99_s=p99)
