"""The allocation-free preconditioner entry point against the context-based one.

pdg_precondition_static serves callers that may not allocate device memory (a budget
fixed at start-up, a host allocator that must not be re-entered, an allocation-free hot
path); it keeps its scratch in a fixed device array instead.  Here it must give the same
result as pdg_precondition (which uses a context and a temporary buffer) on several calls in
a row with different sizes, smoothness weights and inputs, so that no call can lean on what
the one before left in the shared array: a 64^3 call with lambda = 8 first (its z-solve
pivots converge slowly, which sets the array's slow-pivot flag), then 1^3 (no transform at
all: the identity), 2^3 (the middle pivot row is also the last row), 8^3 and 32^3.  This
file is collected last and also runs on its own.
"""
import ctypes as C

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


def test_static_entry_point_matches_context_entry_point_call_after_call():
    import torch

    from paper_2509_18097_gb300 import binding as B

    dev = torch.device("cuda")
    r = np.random.Generator(np.random.PCG64(21))
    for n, lam in ((64, 8.0), (1, 0.5), (2, 0.7), (8, 0.3), (32, 0.5625), (64, 0.84375)):
        g = r.standard_normal((n**3, 3)).astype(np.float32)
        if n > 2:
            g[r.random(n**3) < 0.6] = 0.0
        gd = torch.from_numpy(g).to(dev)
        out = torch.full((n**3, 3), float("nan"), device=dev)
        st = B.pdg_precondition_static(n, lam, gd, out)
        assert st == B.OK
        torch.cuda.synchronize()
        ref = reference(B, n, lam, g)
        got = out.cpu().numpy()
        H.check_close(f"static vs context n={n} lambda={lam}", got, ref)
        if n == 1:  # a single vertex: L = 0, the operator is the identity
            np.testing.assert_array_equal(got, g)


def test_static_entry_point_rejects_what_it_cannot_hold():
    import torch

    from paper_2509_18097_gb300 import binding as B

    dev = torch.device("cuda")
    big = torch.zeros((128**3, 3), device=dev)
    assert B.pdg_precondition_static(128, 0.5, big, torch.empty_like(big)) == B.ERR_BUDGET
    small = torch.zeros((48**3, 3), device=dev)
    assert B.pdg_precondition_static(48, 0.5, small, torch.empty_like(small)) == B.ERR_INVALID  # not a power of two
    # host memory, through the C entry point itself (the wrapper refuses it earlier)
    host = np.zeros((8**3, 3), np.float32)
    lib = B.load()
    st = lib.pdg_precondition_static(8, C.c_float(0.5), host.ctypes.data, np.empty_like(host).ctypes.data, None)
    assert st == B.ERR_INVALID
    # the wrapper checks what the C call cannot: lengths and the device
    with pytest.raises(ValueError):
        B.pdg_precondition_static(8, 0.5, torch.zeros((8**3 - 1, 3), device=dev), torch.zeros((8**3, 3), device=dev))
    with pytest.raises(ValueError):
        B.pdg_precondition_static(8, 0.5, torch.zeros((8**3, 3)), torch.zeros((8**3, 3)))
