"""Host-side checks of the C-ABI library (no GPU needed, no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ctm.h")
LIB = os.path.join(ROOT, "paper_2004_08669_gb300", "libctm_gb300.so")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ctm_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2004_08669_gb300 import build
    build.build()
    return LIB


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("ctm_init", "ctm_step", "ctm_observables", "ctm_step_backward", "ctm_destroy"):
        assert name in syms


def test_library_exports_every_declared_symbol(built_lib):
    lib = ctypes.CDLL(built_lib)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_loads_and_validates_without_gpu(built_lib):
    """Validation runs on the host: bad configurations fail before any CUDA call."""
    import numpy as np

    from paper_2004_08669_gb300 import ctm, workloads as W
    cfg, keep = ctm.make_config(W.dodecahedron(), 8, 2.0)
    assert ctm.ctm_workspace_size(cfg) > 8 * 160 * 160
    bad, keep2 = ctm.make_config(W.dodecahedron() * 1.01, 8, 2.0)
    with pytest.raises(ctm.CtmError) as e:
        ctm.ctm_workspace_size(bad)
    assert e.value.status == ctm.CTM_EINVAL
    neg, keep3 = ctm.make_config(W.dodecahedron(), 8, -1.0)
    with pytest.raises(ctm.CtmError):
        ctm.ctm_workspace_size(neg)
    zero_m, keep4 = ctm.make_config(W.ising(), 0, 1.0)
    with pytest.raises(ctm.CtmError):
        ctm.ctm_workspace_size(zero_m)
    bspin, keep5 = ctm.make_config(W.ising(), 4, 1.0, boundary_spin=2)
    with pytest.raises(ctm.CtmError):
        ctm.ctm_workspace_size(bspin)
    nan_b, keep6 = ctm.make_config(W.ising(), 4, float("nan"))
    with pytest.raises(ctm.CtmError):
        ctm.ctm_workspace_size(nan_b)
    del keep, keep2, keep3, keep4, keep5, keep6, np


def test_host_side_validation_of_the_newer_entry_points(built_lib):
    """The autotuner table, the scan and the correlation length validate
    their arguments on the host, before any CUDA call."""
    from paper_2004_08669_gb300 import ctm, workloads as W
    with pytest.raises(ctm.CtmError) as e:
        ctm.ctm_tc_plan_set("tf32", 64, 64, 64, 96, 1)
    assert e.value.status == ctm.CTM_EINVAL
    with pytest.raises(ctm.CtmError):
        ctm.ctm_tc_plan_set("fp64", 64, 64, 64, 64, 1)
    with pytest.raises(ctm.CtmError):
        ctm.ctm_tc_plan_set("bf16", 64, 64, 64, 128, 17)
    # a pinned shape is read back as the slices it launches (K = 384: six
    # 64-wide K-tiles, three slices of two; K = 200: four tiles, so a request
    # for three gives two slices of two, none empty); clearing restores the
    # default (no split)
    ctm.ctm_tc_plan_set("bf16", 96, 80, 384, 64, 3)
    assert ctm.ctm_tc_plan_get("bf16", 96, 80, 384) == (64, 3)
    ctm.ctm_tc_plan_set("bf16", 96, 80, 200, 64, 3)
    assert ctm.ctm_tc_plan_get("bf16", 96, 80, 200) == (64, 2)
    for K in (384, 200):
        ctm.ctm_tc_plan_set("bf16", 96, 80, K, 0, 0)
        assert ctm.ctm_tc_plan_get("bf16", 96, 80, K)[1] == 1
    cfg, keep = ctm.make_config(W.dodecahedron(), 8, 0.0, prec="tf32")
    one = ctm.ctm_workspace_size(cfg)
    assert ctm.ctm_scan_workspace_size(cfg, 5) >= 5 * one
    with pytest.raises(ctm.CtmError) as e:
        ctm.ctm_scan_init(cfg, [], 2)
    assert e.value.status == ctm.CTM_EINVAL
    with pytest.raises(ctm.CtmError):
        ctm.ctm_scan_init(cfg, [2.0, float("inf")], 2)
    with pytest.raises(ctm.CtmError):
        ctm.ctm_scan_init(cfg, [2.0], 65)
    cfg.workspace = 1 << 40  # never touched: the size check fails first
    cfg.workspace_bytes = 64
    with pytest.raises(ctm.CtmError) as e:
        ctm.ctm_scan_init(cfg, [2.0, 2.5], 2)
    assert e.value.status == ctm.CTM_ENOMEM
    assert ctm.lib.ctm_xi(None, 0, 0.0, None) == ctm.CTM_EINVAL
    assert ctm.lib.ctm_tune(None, 0, None, 0, None) == ctm.CTM_EINVAL
    assert ctm.lib.ctm_scan_run(None, 1, None, None) == ctm.CTM_EINVAL
    assert ctm.lib.ctm_tangent_step(None, None, None, 1, None) == ctm.CTM_EINVAL
    del keep
