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


def test_struct_layouts_match_header():
    import ctypes as C
    import paper_1910_01946_gb300 as pkg
    assert C.sizeof(pkg.rve_options) == 4 * 8 + 11 * 4 + 4   # eleven int32 fields and tail padding
    assert C.sizeof(pkg.rve_material) == 7 * 8 + 6 * 8 + 8 + 5 * 8 + 8
    assert pkg.rve_step_info.local_iters_total.offset == 32 and pkg.rve_step_info.residual.offset == 48
