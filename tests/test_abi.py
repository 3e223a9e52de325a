"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hytg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w]+\s*\*?\s*(hytg_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("hytg_create", "hytg_destroy", "hytg_load_csr", "hytg_set_device_budget",
              "hytg_run", "hytg_fetch_result", "hytg_set_param", "hytg_get_stats",
              "hytg_plan", "hytg_probe_link", "hytg_status_str"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2208_14935_gb300 import build, hytg
    build.build()
    lib = ctypes.CDLL(hytg.LIB_PATH)
    for n in declared_functions():
        assert hasattr(lib, n), n
    hytg.load()
    assert lib  # loads without a GPU


def test_status_strings_without_gpu():
    from paper_2208_14935_gb300 import hytg
    lib = hytg.load()
    assert lib.hytg_status_str(0) == b"ok"
    assert lib.hytg_status_str(3) == b"device budget too small"
    assert lib.hytg_status_str(99) == b"unknown status"


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2208_14935_gb300 import hytg
    saved = hytg._lib
    try:
        hytg._lib = None
        with pytest.raises(hytg.HytgError):
            hytg.load(str(tmp_path / "missing.so"))
    finally:
        hytg._lib = saved
