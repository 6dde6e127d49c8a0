"""Thin ctypes binding of libpdg (include/pdg.h): the same entry-point names, argument
marshalling only.  Every computation runs in the library's CUDA kernels.

Array arguments may be torch tensors (CUDA or CPU; CPU tensors and numpy arrays are
host memory, which the library copies) and are checked for dtype, shape and
contiguity here.  Streams default to torch's current CUDA stream.  The library is loaded
from this package directory; if it is missing, `load()` raises instead of falling back.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpdg.so")
MAX_LEVELS = 8

PAYLOAD_DISPLACEMENT, PAYLOAD_CAYLEY = 0, 1
OK, ERR_INVALID, ERR_OOM, ERR_BUDGET, ERR_CUDA, ERR_NONFINITE, ERR_TIMEOUT, ERR_STATE = range(8)
(BUF_THETA, BUF_GRAD, BUF_PGRAD, BUF_Y, BUF_POINT_GRAD, BUF_NN_FWD, BUF_NN_REV, BUF_LOSS, BUF_SOURCE, BUF_COUNTERS,
 BUF_MESH_GRAD, BUF_MESH_PGRAD) = range(12)
MESH_LAMBDA, MESH_LR = 16.0, 1e-4  # the paper's mesh smoothness weight and learning rate
DEBUG_KEEP_PGRAD, DEBUG_COUNT_NN = 1, 2


class pdg_config(C.Structure):
    _fields_ = [
        ("n_levels", C.c_int),
        ("res", C.c_int * MAX_LEVELS),
        ("lo", C.c_float * 3),
        ("hi", C.c_float * 3),
        ("alpha", C.c_float),
        ("w_chamfer_mesh", C.c_float),
        ("w_chamfer_pts", C.c_float),
        ("w_iso", C.c_float),
        ("lr0", C.c_float),
        ("lr_growth", C.c_float),
        ("lambda0", C.c_float),
        ("lambda_growth", C.c_float),
        ("beta1", C.c_float),
        ("beta2", C.c_float),
        ("eps", C.c_float),
        ("precondition", C.c_int),
        ("robust_weight_stopgrad", C.c_int),
        ("warm_start", C.c_int),
        ("payload", C.c_int),
    ]


class pdg_fit_stats(C.Structure):
    _fields_ = [
        ("loss_total", C.c_double),
        ("cd_mesh", C.c_double),
        ("cd_pts", C.c_double),
        ("iso", C.c_double),
        ("n_steps", C.c_int),
        ("status", C.c_int),
        ("nn_ties", C.c_int),
    ]


class PdgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libpdg status {status}: {msg}")
        self.status = status


_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "pdg_config_default": (None, [C.POINTER(pdg_config)]),
    "pdg_query_bytes": (C.c_size_t, [C.POINTER(pdg_config), C.c_int, C.c_int, C.c_int]),
    "pdg_create": (C.c_int, [C.POINTER(pdg_config), C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_int,
                             C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]),
    "pdg_begin_frame": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "pdg_step": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "pdg_end_frame": (C.c_int, [C.c_void_p, C.POINTER(pdg_fit_stats), C.c_void_p]),
    "pdg_fit_frame": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.POINTER(pdg_fit_stats), C.c_void_p]),
    "pdg_deform": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "pdg_get_vertices": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "pdg_read": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_size_t, C.c_void_p]),
    "pdg_write_theta": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "pdg_set_debug": (C.c_int, [C.c_void_p, C.c_int]),
    "pdg_precondition": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pdg_eval": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_void_p]),
    "pdg_fit_mesh": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_float, C.c_float, C.POINTER(pdg_fit_stats),
                               C.c_void_p]),
    "pdg_precondition_static": (C.c_int, [C.c_int, C.c_float, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pdg_profile_stages": (C.c_int, []),
    "pdg_profile_stage_name": (C.c_char_p, [C.c_int]),
    "pdg_profile_step": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_void_p]),
    "pdg_step_kernel_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "pdg_destroy": (None, [C.c_void_p]),
    "pdg_debug_fail_allocations": (None, [C.c_int]),
    "pdg_status_string": (C.c_char_p, [C.c_int]),
    "pdg_last_error": (C.c_char_p, [C.c_void_p]),
    "pdg_batch_create": (C.c_int, [C.c_int, C.POINTER(C.c_void_p)]),
    "pdg_batch_set": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.c_int]),
    "pdg_batch_step": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "pdg_batch_destroy": (None, [C.c_void_p]),
    "pdg_state_bytes": (C.c_size_t, [C.c_void_p]),
    "pdg_save_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "pdg_load_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
}


def load(path: str = LIB_PATH):
    """Loads libpdg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libpdg.so not found at {path}; run paper_2509_18097_gb300.build.build() first")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


# ---------------------------------------------------------------------------------- marshalling


def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    import torch

    if torch.cuda.is_available():
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(0)


class _Arr:
    """Keeps an array alive and exposes its pointer."""

    def __init__(self, a, dtype, cols=None, name="array"):
        import torch

        if isinstance(a, torch.Tensor):
            want = {np.float32: torch.float32, np.int32: torch.int32}[dtype]
            if a.dtype != want:
                raise TypeError(f"{name} must be {want}, got {a.dtype}")
            if not a.is_contiguous():
                raise ValueError(f"{name} must be contiguous")
            self.obj = a
            self.ptr = a.data_ptr()
            self.n = a.shape[0] if a.dim() else 0
            shape = tuple(a.shape)
        else:
            arr = np.ascontiguousarray(a, dtype=dtype)
            self.obj = arr
            self.ptr = arr.ctypes.data
            self.n = arr.shape[0] if arr.ndim else 0
            shape = arr.shape
        if cols is not None and (len(shape) != 2 or shape[1] != cols):
            raise ValueError(f"{name} must have shape [n, {cols}], got {shape}")


def _check(status: int, ctx=None):
    if status != OK:
        lib = load()
        msg = lib.pdg_last_error(ctx).decode() if ctx else lib.pdg_status_string(status).decode()
        if not msg:
            msg = lib.pdg_status_string(status).decode()
        raise PdgError(status, msg)


# ---------------------------------------------------------------------------------- entry points


def pdg_config_default(**overrides) -> pdg_config:
    cfg = pdg_config()
    load().pdg_config_default(C.byref(cfg))
    for k, v in overrides.items():
        if k == "res":
            cfg.n_levels = len(v)
            for i, n in enumerate(v):
                cfg.res[i] = int(n)
        elif k in ("lo", "hi"):
            for i in range(3):
                getattr(cfg, k)[i] = float(v[i])
        elif k in ("precondition", "robust_weight_stopgrad", "warm_start"):
            setattr(cfg, k, int(bool(v)))
        elif k == "payload":
            cfg.payload = {"displacement": PAYLOAD_DISPLACEMENT, "cayley": PAYLOAD_CAYLEY}.get(v, v)
        else:
            setattr(cfg, k, float(v))
    return cfg


def pdg_query_bytes(cfg: pdg_config, n_verts: int, n_edges: int, max_pts: int) -> int:
    return int(load().pdg_query_bytes(C.byref(cfg), n_verts, n_edges, max_pts))


def pdg_create(cfg: pdg_config, template, edges, source, max_pts: int | None = None, stream=None) -> C.c_void_p:
    lib = load()
    t = _Arr(template, np.float32, 3, "template")
    e = _Arr(edges, np.int32, 2, "edges")
    s = _Arr(source, np.float32, 3, "source")
    mp = int(max_pts if max_pts is not None else s.n)
    out = C.c_void_p()
    st = lib.pdg_create(C.byref(cfg), t.ptr, t.n, e.ptr if e.n else None, e.n, s.ptr, s.n, mp, _stream(stream),
                        C.byref(out))
    _check(st)
    return out


def pdg_begin_frame(ctx, target, stream=None):
    a = _Arr(target, np.float32, 3, "target")
    _check(load().pdg_begin_frame(ctx, a.ptr, a.n, _stream(stream)), ctx)


def pdg_step(ctx, n_steps: int = 1, stream=None):
    _check(load().pdg_step(ctx, int(n_steps), _stream(stream)), ctx)


def pdg_end_frame(ctx, stream=None) -> pdg_fit_stats:
    st = pdg_fit_stats()
    _check(load().pdg_end_frame(ctx, C.byref(st), _stream(stream)), ctx)
    return st


def pdg_fit_frame(ctx, target, n_steps: int, stream=None) -> pdg_fit_stats:
    a = _Arr(target, np.float32, 3, "target")
    st = pdg_fit_stats()
    _check(load().pdg_fit_frame(ctx, a.ptr, a.n, int(n_steps), C.byref(st), _stream(stream)), ctx)
    return st


def pdg_deform(ctx, xyz, out, stream=None):
    a = _Arr(xyz, np.float32, 3, "xyz")
    o = _Arr(out, np.float32, 3, "out")
    if o.n != a.n:
        raise ValueError("out must have the same number of points as xyz")
    _check(load().pdg_deform(ctx, a.ptr, a.n, o.ptr, _stream(stream)), ctx)
    return out


def pdg_get_vertices(ctx, out, stream=None):
    o = _Arr(out, np.float32, 3, "out")
    _check(load().pdg_get_vertices(ctx, o.ptr, _stream(stream)), ctx)
    return out


def pdg_read(ctx, which: int, level: int, out, stream=None):
    import torch

    if isinstance(out, torch.Tensor):
        ptr, nbytes = out.data_ptr(), out.numel() * out.element_size()
    else:
        ptr, nbytes = out.ctypes.data, out.nbytes
    _check(load().pdg_read(ctx, int(which), int(level), ptr, nbytes, _stream(stream)), ctx)
    return out


def pdg_write_theta(ctx, level: int, theta, stream=None):
    a = _Arr(theta, np.float32, None, "theta")  # [res^3, C]; the library checks nothing else
    _check(load().pdg_write_theta(ctx, int(level), a.ptr, _stream(stream)), ctx)


def pdg_eval(ctx, stream=None) -> np.ndarray:
    """Loss (total, cd_mesh, cd_pts, iso) and gradients at the current grids, no update."""
    out = (C.c_double * 4)()
    _check(load().pdg_eval(ctx, out, _stream(stream)), ctx)
    return np.array(out[:], np.float64)


def pdg_fit_mesh(ctx, p0, n_steps: int, lam: float = MESH_LAMBDA, lr: float = MESH_LR, stream=None) -> pdg_fit_stats:
    """Template-mesh fit of the context's vertices to the keyframe cloud p0 [n, 3]."""
    a = _Arr(p0, np.float32, 3, "p0")
    st = pdg_fit_stats()
    _check(load().pdg_fit_mesh(ctx, a.ptr, a.n, int(n_steps), float(lam), float(lr), C.byref(st), _stream(stream)), ctx)
    return st


def pdg_precondition(ctx, level: int, g, out, stream=None):
    a = _Arr(g, np.float32, 3, "g")
    o = _Arr(out, np.float32, 3, "out")
    _check(load().pdg_precondition(ctx, int(level), a.ptr, o.ptr, _stream(stream)), ctx)
    return out


def pdg_precondition_static(res: int, lam: float, g, out, stream=None):
    """Allocation-free (I + lambda L)^{-2} on a res^3 grid; g and out must be float32 CUDA
    tensors of shape [res^3, 3] on the current device (ValueError otherwise: the C entry
    point cannot check a buffer's length).  Returns the status code of the call (not raised:
    callers of this entry point typically handle errors themselves)."""
    import torch

    for name, t in (("g", g), ("out", out)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} must be on the current device cuda:{torch.cuda.current_device()}")
    a = _Arr(g, np.float32, 3, "g")
    o = _Arr(out, np.float32, 3, "out")
    if res >= 1 and not (a.n == o.n == int(res) ** 3):
        raise ValueError(f"g and out must hold res^3 = {int(res) ** 3} rows, got {a.n} and {o.n}")
    return int(load().pdg_precondition_static(int(res), float(lam), a.ptr, o.ptr, _stream(stream)))


def pdg_set_debug(ctx, keep_pgrad: bool = True, count_nn: bool = False):
    flags = (DEBUG_KEEP_PGRAD if keep_pgrad else 0) | (DEBUG_COUNT_NN if count_nn else 0)
    _check(load().pdg_set_debug(ctx, flags), ctx)


def pdg_debug_fail_allocations(n: int):
    """Test hook: the library's next n device allocations fail (PDG_ERR_OOM)."""
    load().pdg_debug_fail_allocations(int(n))


def pdg_profile_stages() -> int:
    return int(load().pdg_profile_stages())


def pdg_profile_stage_name(i: int) -> str:
    return load().pdg_profile_stage_name(int(i)).decode()


def pdg_profile_step(ctx, n_steps: int, stream=None) -> dict:
    """Eager, event-bracketed iterations; returns {stage name: total ms}."""
    n = pdg_profile_stages()
    buf = (C.c_double * n)()
    _check(load().pdg_profile_step(ctx, int(n_steps), buf, _stream(stream)), ctx)
    return {pdg_profile_stage_name(i): buf[i] for i in range(n)}


def pdg_step_kernel_count(ctx) -> int:
    """Kernel launches per pdg_step iteration (0 before the first step)."""
    out = C.c_int(0)
    _check(load().pdg_step_kernel_count(ctx, C.byref(out)), ctx)
    return int(out.value)


def pdg_destroy(ctx):
    if ctx:
        load().pdg_destroy(ctx)


def pdg_status_string(status: int) -> str:
    return load().pdg_status_string(int(status)).decode()


def pdg_last_error(ctx) -> str:
    return load().pdg_last_error(ctx).decode()


def pdg_batch_create(max_jobs: int) -> C.c_void_p:
    out = C.c_void_p()
    _check(load().pdg_batch_create(int(max_jobs), C.byref(out)))
    return out


def pdg_batch_set(batch, ctxs):
    arr = (C.c_void_p * max(len(ctxs), 1))(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])
    _check(load().pdg_batch_set(batch, arr, len(ctxs)))


def pdg_batch_step(batch, n_steps: int = 1, stream=None):
    _check(load().pdg_batch_step(batch, int(n_steps), _stream(stream)))


def pdg_batch_destroy(batch):
    if batch:
        load().pdg_batch_destroy(batch)


def pdg_state_bytes(ctx) -> int:
    return int(load().pdg_state_bytes(ctx))


def pdg_save_state(ctx, stream=None) -> bytes:
    n = pdg_state_bytes(ctx)
    buf = C.create_string_buffer(n)
    _check(load().pdg_save_state(ctx, buf, n, _stream(stream)), ctx)
    return buf.raw


def pdg_load_state(ctx, data: bytes, stream=None):
    buf = C.create_string_buffer(data, len(data))
    _check(load().pdg_load_state(ctx, buf, len(data), _stream(stream)), ctx)
