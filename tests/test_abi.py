"""The C ABI library loads and exports every entry point declared in
include/aw.h; the Python binding names the same functions (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "aw.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|char\s*\*|const\s+char\s*\*)\s*\*?\s*(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2206_15117_gb300 import aw, build
    build.build()
    return aw.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["aw_make_kernels", "aw_grid", "aw_degrid", "aw_fft_to_image", "mosaic_gamma",
                     "aw_plan_create", "aw_grid_batched", "aw_autotune"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib):
    from paper_2206_15117_gb300 import aw
    assert set(declared_functions()) == set(aw.SIGNATURES)


def test_struct_sizes_match_header_layout(lib):
    import ctypes
    from paper_2206_15117_gb300 import aw
    # natural C layout on LP64: checked against the field order of the header
    assert ctypes.sizeof(aw.aw_tune) == 20
    assert ctypes.sizeof(aw.aw_stats) == 40
    assert ctypes.sizeof(aw.aw_vis_desc) == 8 * 3 + 8 * 8
    assert ctypes.sizeof(aw.aw_plan_info) == 5 * 8 + 8 + 8 + 8


def test_last_error_is_empty_string_initially(lib):
    assert lib.aw_last_error() in (b"",) or isinstance(lib.aw_last_error(), bytes)
