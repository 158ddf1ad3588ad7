"""The C ABI library builds for sm_103a, loads, and exports every entry point
that include/rve.h declares; host-only entry points answer without a GPU."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1910_01946_gb300 import _build
    _build.build()
    import paper_1910_01946_gb300 as pkg
    return pkg.load_library()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rve.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rve_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    import paper_1910_01946_gb300 as pkg
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(pkg.EXPORTED)


def test_workspace_bytes_validation(lib):
    import paper_1910_01946_gb300 as pkg
    assert pkg.rve_workspace_bytes(16, 16, 16, 8) > 0
    assert pkg.rve_workspace_bytes(48, 96, 9, 100) > 0
    assert pkg.rve_workspace_bytes(15, 16, 16, 8) == 0      # odd n0
    assert pkg.rve_workspace_bytes(16, 16, 10, 8) == 0      # 10 = 2 * 5
    assert pkg.rve_workspace_bytes(16, 16, 16, 0) == 0
    assert pkg.rve_workspace_bytes(16, 16, 16, 8, 7) == 0   # unknown precision
    small = pkg.rve_workspace_bytes(32, 32, 32, 8)
    big = pkg.rve_workspace_bytes(64, 64, 64, 8)
    assert 7.5 * small < big < 8.5 * small


def test_struct_layouts_match_header(tmp_path):
    """Every field offset and the size of each struct shared with the binding,
    as the C compiler lays them out from include/rve.h, equal the ctypes
    layout the binding uses."""
    import ctypes as C
    import shutil
    import subprocess
    import paper_1910_01946_gb300 as pkg
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"rve_options": pkg.rve_options, "rve_material": pkg.rve_material, "rve_step_info": pkg.rve_step_info}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "rve.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            name, field, val = ln.split()
            got[(name, field)] = int(val)
    for name, cls in structs.items():
        assert got[(name, "sizeof")] == C.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)
