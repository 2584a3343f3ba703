"""CPU-only checks of the boundary: the CUDA library builds, loads and exports every
entry point that include/bgk.h declares (no compute calls without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "bgk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bgk_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ["bgk_create", "bgk_destroy", "bgk_step", "bgk_sweep", "bgk_get_moments", "bgk_get_generations",
                 "bgk_set_state_maxwellian", "bgk_set_inflow_maxwellian", "bgk_status_string"]:
        assert must in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2608_19150_b300 import build as B
    path = B.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    from paper_2608_19150_b300 import bgk
    lib = bgk.load()
    assert lib.bgk_status_string(0) == b"ok"
    assert b"converge" in lib.bgk_status_string(4)


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2608_19150_b300 import bgk
    saved = bgk._lib
    bgk._lib = None
    try:
        with pytest.raises(RuntimeError):
            bgk.load(str(tmp_path / "missing.so"))
    finally:
        bgk._lib = saved
