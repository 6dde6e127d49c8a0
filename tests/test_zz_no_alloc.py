"""The allocation-free preconditioner entry point against the context-based one.

pdg_precondition_static serves callers that may not allocate device memory (a budget
fixed at start-up, a host allocator that must not be re-entered, an allocation-free hot
path); it keeps its scratch in a fixed device array instead.  Here it must give the same
result as pdg_precondition (which uses a context and a temporary buffer) on two calls in a
row with different sizes and inputs, so that the second call cannot lean on what the
first left in the shared array.  This file is collected last and also runs on its own.
"""
import numpy as np
import pytest

from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def reference(B, n, lam, g):
    v = np.zeros((1, 3), np.float32)
    ctx = B.pdg_create(B.pdg_config_default(res=(n,), lambda0=lam), v, np.zeros((0, 2), np.int32), v, max_pts=1)
    try:
        return B.pdg_precondition(ctx, 0, g, np.empty_like(g))
    finally:
        B.pdg_destroy(ctx)


def test_static_entry_point_matches_context_entry_point_twice():
    import torch

    from paper_2509_18097_gb300 import binding as B

    dev = torch.device("cuda")
    r = np.random.Generator(np.random.PCG64(21))
    for n, lam in ((64, 0.84375), (32, 0.5625)):
        g = r.standard_normal((n**3, 3)).astype(np.float32)
        g[r.random(n**3) < 0.6] = 0.0
        gd = torch.from_numpy(g).to(dev)
        out = torch.full((n**3, 3), float("nan"), device=dev)
        st = B.pdg_precondition_static(n, lam, gd, out)
        assert st == B.OK
        torch.cuda.synchronize()
        ref = reference(B, n, lam, g)
        H.check_close(f"static vs context n={n}", out.cpu().numpy(), ref)


def test_static_entry_point_rejects_what_it_cannot_hold():
    import torch

    from paper_2509_18097_gb300 import binding as B

    dev = torch.device("cuda")
    big = torch.zeros((128**3, 3), device=dev)
    assert B.pdg_precondition_static(128, 0.5, big, torch.empty_like(big)) == B.ERR_BUDGET
    small = torch.zeros((48**3, 3), device=dev)
    assert B.pdg_precondition_static(48, 0.5, small, torch.empty_like(small)) == B.ERR_INVALID  # not a power of two
    host = np.zeros((8**3, 3), np.float32)
    assert B.pdg_precondition_static(8, 0.5, host, np.empty_like(host)) == B.ERR_INVALID  # host memory
