"""GB300-native (sm_103a) per-iteration step of Preconditioned Deformation Grids.

The compute path is the C-ABI library `libpdg.so` (hand-written CUDA kernels); this
package holds its thin ctypes binding (`binding`), a convenience layer (`api`), the
torch.autograd.Function wrappers (`autograd`), the continuous-batching server (`serve`)
and the seeded synthetic-input generators (`synth`).  Nothing is loaded at import time;
the binding raises if the library is missing.
"""
__all__ = ["synth"]
