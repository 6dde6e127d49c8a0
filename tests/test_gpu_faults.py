"""Failure paths of the C-ABI on the GPU, made on the host side or with valid inputs: no
test here faults, traps or hangs a GPU.

* A non-finite loss: a target point at 3e19 is a finite input, but its squared distance to
  anything overflows FP32, so its robust-Chamfer term is NaN.  The frame must end with
  PDG_ERR_NONFINITE (not a fault), and the context must stay usable.
* An allocation failure: the library's test hook makes its next device allocation fail;
  the call must return PDG_ERR_OOM, free what it had taken, and leave the library working.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2509_18097_gb300 import synth

pytestmark = pytest.mark.gpu


def workload(seed=41):
    r = np.random.Generator(np.random.PCG64(seed))
    v, _, e = synth.icosphere(2)
    src = synth.sphere_points(r, 700).astype(np.float32)
    tgt = synth.sinusoid(synth.sphere_points(r, 800), 0.1).astype(np.float32)
    return v, e, src, tgt, (4, 8, 16)


def test_nonfinite_loss_is_a_status_and_the_context_stays_usable():
    from paper_2509_18097_gb300 import binding as B

    v, e, src, tgt, res = workload()
    ctx = B.pdg_create(B.pdg_config_default(res=res), v, e, src, max_pts=len(tgt))
    fresh = None
    try:
        state0 = B.pdg_save_state(ctx)
        bad = tgt.copy()
        bad[5] = (3e19, 0.1, 0.2)  # finite; its squared distance to any point overflows FP32
        B.pdg_begin_frame(ctx, bad)
        B.pdg_step(ctx, 3)
        stats = B.pdg_fit_stats()
        st = B.load().pdg_end_frame(ctx, C.byref(stats), None)
        assert st == B.ERR_NONFINITE and stats.status == B.ERR_NONFINITE
        assert not np.isfinite(stats.loss_total)
        assert "NaN" in B.pdg_last_error(ctx)
        # usable afterwards: restored to its first state, it fits exactly as a new context does
        B.pdg_load_state(ctx, state0)
        s1 = B.pdg_fit_frame(ctx, tgt, 5)
        x1 = B.pdg_get_vertices(ctx, np.empty((len(v), 3), np.float32))
        fresh = B.pdg_create(B.pdg_config_default(res=res), v, e, src, max_pts=len(tgt))
        s2 = B.pdg_fit_frame(fresh, tgt, 5)
        x2 = B.pdg_get_vertices(fresh, np.empty((len(v), 3), np.float32))
        assert s1.status == B.OK and np.isfinite(s1.loss_total)
        assert s1.loss_total == s2.loss_total
        assert np.array_equal(x1, x2)
    finally:
        B.pdg_destroy(ctx)
        B.pdg_destroy(fresh)


def test_allocation_failure_is_a_status_and_leaks_nothing():
    import torch

    from paper_2509_18097_gb300 import binding as B

    v, e, src, tgt, res = workload(42)
    cfg = B.pdg_config_default(res=res)
    ctx = B.pdg_create(cfg, v, e, src, max_pts=len(tgt))  # warm: library state, kernel attributes
    B.pdg_destroy(ctx)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    try:
        for _ in range(20):
            B.pdg_debug_fail_allocations(1)
            with pytest.raises(B.PdgError) as ei:
                B.pdg_create(cfg, v, e, src, max_pts=len(tgt))
            assert ei.value.status == B.ERR_OOM
            B.pdg_debug_fail_allocations(1)
            with pytest.raises(B.PdgError) as ei:
                B.pdg_batch_create(4)
            assert ei.value.status == B.ERR_OOM
    finally:
        B.pdg_debug_fail_allocations(0)
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= 4 << 20
    # the hook is spent: the library works as before
    ctx = B.pdg_create(cfg, v, e, src, max_pts=len(tgt))
    try:
        s = B.pdg_fit_frame(ctx, tgt, 2)
        assert s.status == B.OK and np.isfinite(s.loss_total)
    finally:
        B.pdg_destroy(ctx)
