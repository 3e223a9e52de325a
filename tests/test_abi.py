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


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the ABI structs have the C compiler's size and
    field offsets (a drift would silently misread statistics)."""
    import subprocess
    from paper_2208_14935_gb300 import hytg
    structs = {"hytg_stats": hytg.hytg_stats, "hytg_info": hytg.hytg_info,
               "hytg_iter_record": hytg.hytg_iter_record, "hytg_cost_params": hytg.hytg_cost_params,
               "hytg_timed_launch": hytg.hytg_timed_launch, "hytg_serve_info": hytg.hytg_serve_info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hytg.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            a, b, c = line.split()
            got[(a, b)] = int(c)
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)
