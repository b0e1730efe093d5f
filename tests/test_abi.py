"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, and
exports every function include/*.h declares; the ctypes descriptor has the C
layout (checked against gcc's own sizeof/offsetof of cr_mesh_desc)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2604_02125_gb300 import build, crkfr
    build.build()
    return crkfr.load_library()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(cr_[A-Za-z0-9_]+)\s*\(", src, re.M):
            names.add(m.group(1))
    return names


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert {"cr_init_mesh", "cr_set_state", "cr_step", "cr_get_state"} <= names
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    from paper_2604_02125_gb300 import crkfr
    for s in (0, -1, -2, -3, -4, -5, -6):
        assert crkfr.status_string(s)
    assert "non-physical" in crkfr.status_string(-4)


def test_null_context_is_rejected_without_gpu(lib):
    # argument checks happen before any CUDA call
    assert lib.cr_step(None, 1) == -1
    assert lib.cr_sync(None) == -1
    assert lib.cr_destroy(None) == -1
    assert lib.cr_init_mesh(None, None, 1, None) == -1


def test_descriptor_layout_matches_c(tmp_path):
    from paper_2604_02125_gb300 import crkfr
    src = tmp_path / "lay.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "cr.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu\\n", sizeof(cr_mesh_desc),'
                   'offsetof(cr_mesh_desc, lo), offsetof(cr_mesh_desc, gamma),'
                   'offsetof(cr_mesh_desc, dt_fixed), offsetof(cr_mesh_desc, prec)); return 0;}\n')
    exe = tmp_path / "lay"
    subprocess.check_call(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    D = crkfr.MeshDesc
    assert got == [ctypes.sizeof(D), D.lo.offset, D.gamma.offset, D.dt_fixed.offset, D.prec.offset]
