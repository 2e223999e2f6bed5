"""The C ABI library loads and exports every entry point declared in
include/aw.h; the Python binding names the same functions (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")
HEADER = os.path.join(INCLUDE, "aw.h")


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
    assert ctypes.sizeof(aw.aw_tune) == 24
    assert ctypes.sizeof(aw.aw_stats) == 40
    assert ctypes.sizeof(aw.aw_vis_desc) == 8 * 3 + 8 * 8
    assert ctypes.sizeof(aw.aw_plan_info) == 5 * 8 + 8 + 8 + 8 + 8


def test_struct_layout_matches_the_c_compiler(tmp_path):
    # the header compiled as C99 by the host compiler: sizes and field offsets
    import ctypes
    import shutil
    import subprocess
    from paper_2206_15117_gb300 import aw
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"aw_tune": aw.aw_tune, "aw_stats": aw.aw_stats, "aw_vis_desc": aw.aw_vis_desc,
               "aw_plan_info": aw.aw_plan_info}
    lines = []
    for name, cls in structs.items():
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (name, name))
        for fname, _ in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, fname, name, fname))
    src = tmp_path / "abi.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "aw.h"\nint main(void) {\n%s\nreturn 0;\n}\n'
                   % "\n".join(lines))
    exe = tmp_path / "abi"
    subprocess.run([cc, "-std=c99", "-I" + INCLUDE, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name, cls in structs.items():
        assert got[(name, "sizeof")] == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert got[(name, fname)] == getattr(cls, fname).offset, (name, fname)


def test_last_error_is_empty_string_initially(lib):
    assert lib.aw_last_error() in (b"",) or isinstance(lib.aw_last_error(), bytes)
