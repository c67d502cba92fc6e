"""The C ABI library builds, loads and exports every symbol include/fmocc.h declares (no GPU
needed: nothing here launches a kernel)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fmocc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w ]+\*?\s*\**\s*(fm_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    import shutil
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit")
    from paper_1811_06127_gb300 import _build, fmocc
    _build.build()
    return fmocc.load_library()


def test_header_declares_the_calls():
    names = declared_functions()
    for want in ("fm_build", "fm_free", "fm_occ8", "fm_exact", "fm_dcalc", "fm_inexact",
                 "fm_save", "fm_load", "fm_info", "fm_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1811_06127_gb300 import fmocc
    names = declared_functions()
    assert sorted(names) == sorted(fmocc.EXPORTS)
    for name in names:
        assert hasattr(lib, name), name


def test_host_side_argument_errors(lib):
    """Argument validation happens before any device work."""
    import ctypes as C
    from paper_1811_06127_gb300 import fmocc
    out = C.c_void_p()
    p = fmocc.fm_params(64, 0, -1, 0)
    assert lib.fm_build(None, 10, C.byref(p), C.byref(out)) == fmocc.FM_EINVAL
    assert lib.fm_build(C.c_char_p(b"ACGT"), 0, C.byref(p), C.byref(out)) == fmocc.FM_EINVAL
    p.interval = 100
    assert lib.fm_build(C.c_char_p(b"ACGT"), 4, C.byref(p), C.byref(out)) == fmocc.FM_EINVAL
    assert b"interval" in lib.fm_last_error(None)
    # both strands double the text: |R| above 2^30 - 1 is refused before any buffer is read
    p.interval, p.flags = 64, fmocc.FM_BUILD_BOTH_STRANDS
    assert lib.fm_build(C.c_char_p(b"ACGT"), 1073741824, C.byref(p), C.byref(out)) == fmocc.FM_EINVAL
    assert b"BOTH_STRANDS" in lib.fm_last_error(None)
    assert lib.fm_occ8(None, None, None, None, 0, None) == fmocc.FM_EINVAL
    assert lib.fm_inexact(None, None, None, 0, None, None, None, None, 0, None, None) == fmocc.FM_EINVAL


def test_struct_layouts_match_header(tmp_path):
    """Every public struct of include/fmocc.h has, in the ctypes binding, the C compiler's size
    and the same offset for every field (a drift between the two corrupts arguments)."""
    import ctypes
    import shutil
    import subprocess

    from paper_1811_06127_gb300 import fmocc

    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    structs = [fmocc.fm_params, fmocc.fm_info_t, fmocc.fm_profile, fmocc.fm_search_params,
               fmocc.fm_tuning, fmocc.fm_server_params, fmocc.fm_server_result]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fmocc.h"', 'int main(void) {']
    for st in structs:
        name = st.__name__
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in st._fields_:
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ['return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-std=c11", "-I", inc, "-o", str(exe), str(src)], check=True)
    got = dict(line.rsplit(" ", 1) for line in
               subprocess.run([str(exe)], capture_output=True, text=True, check=True)
               .stdout.splitlines())
    for st in structs:
        name = st.__name__
        assert int(got[f"{name} size"]) == ctypes.sizeof(st), name
        for field, _ in st._fields_:
            assert int(got[f"{name} {field}"]) == getattr(st, field).offset, (name, field)
