"""The C-ABI library builds, loads and exports what include/tc.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

import paper_2512_01055_gb300 as tc
from paper_2512_01055_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*[\s\*]+(tc_[a-z_0-9]+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return tc.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "tc_energy" in names and "tc_init" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(tc.EXPORTS)


def test_status_strings(lib):
    assert tc.status_str(tc.TC_OK) == "TC_OK"
    assert tc.status_str(tc.TC_ENOMEM) == "TC_ENOMEM"
    assert tc.status_str(99) == "TC_UNKNOWN"


def test_workspace_bytes_is_host_arithmetic(lib):
    assert tc.tc_workspace_bytes(0, 10) == 0
    a = tc.tc_workspace_bytes(6, 36)
    b = tc.tc_workspace_bytes(20, 200)
    assert 0 < a < b


def test_null_context_is_rejected(lib):
    res = tc.tc_result()
    ints = tc.tc_ints()
    assert lib.tc_energy(None, 2, 2, None, None, None, ctypes.byref(ints), 0, 0, None, ctypes.byref(res)) == tc.TC_EINVAL
    lib.tc_finalize(None)
    assert lib.tc_last_error(None) == b""


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes structures of the binding have the sizes and field offsets of include/tc.h (compiled with cc)."""
    import shutil
    import subprocess
    cc = shutil.which("cc") or shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [tc.tc_options, tc.tc_ints, tc.tc_job, tc.tc_serve_stats, tc.tc_result]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "tc.h"', "int main(void) {"]
    for st in structs:
        n = st.__name__
        lines.append(f'  printf("{n} %zu\\n", sizeof({n}));')
        for f, _ in st._fields_:
            lines.append(f'  printf("{n}.{f} %zu\\n", offsetof({n}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.splitlines())
    for st in structs:
        n = st.__name__
        assert int(got[n]) == ctypes.sizeof(st), n
        for f, _ in st._fields_:
            assert int(got[f"{n}.{f}"]) == getattr(st, f).offset, f"{n}.{f}"
