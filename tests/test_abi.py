"""The C-ABI library builds for sm_103a, loads, and exports every function
include/rgrt.h declares.  CPU only: no compute call is made."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "rgrt.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                       text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "return")))


@pytest.fixture(scope="module")
def lib():
    from paper_2602_01057_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_five_calls():
    names = _declared_functions()
    for n in ("gaussians_create", "geometry_set", "project_forward", "project_backward", "loss_step"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2602_01057_gb300 import rgrt
    assert set(_declared_functions()) <= set(rgrt.exported_symbols())


def test_last_error_is_empty_string_initially(lib):
    lib.rgrt_last_error.restype = ctypes.c_char_p
    assert lib.rgrt_last_error() in (b"",)


def test_null_arguments_are_rejected_without_a_device(lib):
    from paper_2602_01057_gb300 import rgrt
    L = rgrt.lib()
    assert L.rgrt_ctx_create(None, 0, 0) == -1        # RGRT_E_INVAL
    assert L.project_forward(None, None, None, None, None) == -1
    assert b"null" in L.rgrt_last_error()


def _c_layout(struct, fields, tmp_path):
    """sizeof and offsetof of a header struct, from a C program compiled here."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rgrt.h"', 'int main(void) {',
             f'  printf("%zu\\n", sizeof({struct}));']
    lines += [f'  printf("%zu\\n", offsetof({struct}, {f}));' for f in fields]
    lines += ['  return 0;', '}']
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    return int(out[0]), [int(x) for x in out[1:]]


@pytest.mark.parametrize("struct,cls", [("rgrt_geom_desc", "GeomDesc"), ("rgrt_adam", "Adam"),
                                        ("rgrt_volume_desc", "VolumeDesc")])
def test_binding_structs_match_the_header(struct, cls, tmp_path):
    """The ctypes mirrors of the descriptor structs have the header's field
    order, offsets and size."""
    from paper_2602_01057_gb300 import rgrt
    C = getattr(rgrt, cls)
    names = [f[0] for f in C._fields_]
    size, offs = _c_layout(struct, names, tmp_path)
    assert ctypes.sizeof(C) == size
    assert [getattr(C, n).offset for n in names] == offs
