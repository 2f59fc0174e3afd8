"""The CUDA library builds, loads on the CPU host and exports every entry point that
include/vecchia.h declares (no compute calls: this host has no GPU)."""
import ctypes
import os
import re

import pytest

import paper_2407_02740_gb300 as vg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"VECCHIA_API\s+[\w\s\*]*?\b(vecchia_\w+)\s*\(", src))
    return names


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("vecchia_loglik_grad_info", "vecchia_loglik_grad_info_host",
                     "vecchia_create", "vecchia_destroy", "vecchia_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    if not os.path.exists(vg.LIB_PATH):
        vg.build()
    lib = ctypes.CDLL(vg.LIB_PATH)
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_host_only_queries_and_argument_errors():
    lib = vg.lib()
    assert lib.vecchia_nparms(vg.EXP_ISO) == 3
    assert lib.vecchia_nparms(vg.MATERN_ISO) == 4
    assert lib.vecchia_nparms(vg.EXP_SPACETIME) == 4
    assert lib.vecchia_nparms(99) == -1
    assert lib.vecchia_nparms(vg.EXP_ANISO) == -1          # depends on d
    assert lib.vecchia_nparms_d(vg.EXP_ANISO, 18) == 20
    assert lib.vecchia_nparms_d(vg.EXP_ANISO, 21) == -1
    assert lib.vecchia_nparms_d(vg.EXP_ISO, 4) == -1
    assert lib.vecchia_nparms_d(vg.EXP_SPACETIME, 2) == -1
    assert lib.vecchia_nparms_d(vg.MATERN_ISO, 2) == 4
    assert lib.vecchia_max_m() >= 60
    # a NULL handle or plan is rejected before any CUDA call
    assert lib.vecchia_set_lanes(None, 4) == 1
    assert b"NULL" in lib.vecchia_last_error()
    assert lib.vecchia_set_group_chunk(None, 4) == 1
    assert lib.vecchia_batch_plan_class(None, 0, None, None, None, None) == 1
    assert lib.vecchia_kernels_per_pass(vg.MATERN_ISO) == 5
    assert lib.vecchia_kernels_per_pass(99) == -1


def test_no_fallback_without_the_library(monkeypatch, tmp_path):
    # the product path has no CPU fallback: without the built library every call fails loudly
    monkeypatch.setattr(vg, "_lib", None)
    monkeypatch.setattr(vg, "LIB_PATH", str(tmp_path / "libvecchia_gb300.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        vg.lib()
    with pytest.raises(RuntimeError):
        vg.nparms(vg.EXP_ISO, 2)
