"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads, exports every
entry point declared in include/pdg.h, and its host-only calls behave as documented."""
import ctypes as C
import json
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2509_18097_gb300 import binding, build

    build.build()
    return binding.load()


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(pdg_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_entry_point():
    from paper_2509_18097_gb300 import binding

    missing = [n for n in declared_functions() if not hasattr(binding, n)]
    assert not missing, missing


def test_config_default_is_the_papers(lib):
    from paper_2509_18097_gb300 import binding

    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))
    c = binding.pdg_config_default()
    f32 = lambda v: C.c_float(v).value
    assert c.alpha == f32(g["alpha"]["value"])
    assert c.w_iso == f32(g["w_isometry"]["value"])
    assert c.lr0 == f32(g["lr0"]["value"]) and c.lr_growth == f32(g["lr_growth"]["value"])
    assert c.lambda0 == f32(g["lambda0"]["value"]) and c.lambda_growth == f32(g["lambda_growth"]["value"])
    assert (c.beta1, c.beta2, c.eps) == tuple(f32(g[k]["value"]) for k in ("beta1", "beta2", "eps"))
    assert c.precondition == 1 and c.robust_weight_stopgrad == 0
    assert c.n_levels == 4 and list(c.res)[:4] == [16, 32, 64, 128]
    assert list(c.lo) == [-1.5] * 3 and list(c.hi) == [1.5] * 3


def test_query_bytes(lib):
    from paper_2509_18097_gb300 import binding

    cfg = binding.pdg_config_default()
    b = binding.pdg_query_bytes(cfg, 50412, 151230, 100000)
    # grids alone: theta (16 B) + m, v, g, tmp (12 B each) per vertex of 16^3..128^3
    verts = 16**3 + 32**3 + 64**3 + 128**3
    assert b > verts * 64
    assert b < 2 * 1024**3
    # resolutions: 1 or 2^a 3^b up to 256 (the line transforms are radix-2/3 FFTs)
    for res in ((16, 48), (3, 9, 27, 81), (24, 96, 192), (1, 2, 256), (6, 18, 54, 162, 216, 243)):
        assert binding.pdg_query_bytes(binding.pdg_config_default(res=res), 10, 10, 10) > 0, res
    for res in ((16, 40), (5,), (7, 14), (256, 288), (0,), (512,)):
        assert binding.pdg_query_bytes(binding.pdg_config_default(res=res), 10, 10, 10) == 0, res
    # the Cayley payload takes plane-path levels only (1 or a power of two up to 128)
    assert binding.pdg_query_bytes(binding.pdg_config_default(res=(16, 48), payload="cayley"), 10, 10, 10) == 0
    assert binding.pdg_query_bytes(binding.pdg_config_default(res=(16, 128), payload="cayley"), 10, 10, 10) > 0
    assert binding.pdg_query_bytes(cfg, 0, 10, 10) == 0


def test_status_strings(lib):
    from paper_2509_18097_gb300 import binding

    assert binding.pdg_status_string(0) == "ok"
    assert "invalid" in binding.pdg_status_string(1)
    assert binding.pdg_status_string(99) == "unknown status"


def test_create_rejects_bad_arguments_without_touching_a_gpu(lib):
    """Argument validation happens before any device call."""
    from paper_2509_18097_gb300 import binding

    cfg = binding.pdg_config_default()
    out = C.c_void_p()
    # n_src > max_pts
    st = lib.pdg_create(C.byref(cfg), None, 10, None, 0, None, 5, 4, None, C.byref(out))
    assert st == binding.ERR_INVALID and not out.value
    bad = binding.pdg_config_default(res=(0,))
    st = lib.pdg_create(C.byref(bad), None, 10, None, 0, None, 5, 5, None, C.byref(out))
    assert st == binding.ERR_INVALID


def test_batched_workload_sizes_are_accepted(lib):
    """The batched / served workload draws its levels as 2^a 3^b sizes: each is one the
    library accepts, the finest lies in the drawn range, and levels do not shrink toward the finest."""
    from paper_2509_18097_gb300 import binding, synth

    assert synth.smooth23(181) == 192 and synth.smooth23(100) == 96 and synth.smooth23(13.5) == 12
    for m in synth.SMOOTH_SIZES:
        k = m
        while k % 2 == 0:
            k //= 2
        while k % 3 == 0:
            k //= 3
        assert k == 1 and 2 <= m <= 256
    for i in range(40):
        res = synth.batched_job(i)["res"]
        assert 27 <= res[-1] <= 256 and all(r >= 4 for r in res)
        assert all(a <= b for a, b in zip(res, res[1:])), res  # the floor of 4 may repeat
        cfg = binding.pdg_config_default(res=res)
        assert binding.pdg_query_bytes(cfg, 10, 10, 10) > 0, res
