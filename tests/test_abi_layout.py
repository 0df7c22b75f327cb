"""The ctypes structures of the Python binding match the C header: a small C program compiled
against include/dmpc.h prints the size and every field offset of dmpc_options and dmpc_ocp_desc,
which must equal the binding's (a field added to one side only shifts every later field)."""
import json
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _c_layout(struct, fields):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "dmpc.h"', "int main(void) {",
             f'  printf("{{\\"size\\": %zu", sizeof({struct}));']
    for f in fields:
        lines.append(f'  printf(", \\"{f}\\": %zu", offsetof({struct}, {f}));')
    lines += ['  printf("}\\n");', "  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(src, "w") as fh:
            fh.write("\n".join(lines))
        subprocess.run([cc, "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True, capture_output=True)
        return json.loads(subprocess.run([exe], check=True, capture_output=True, text=True).stdout)


@pytest.mark.parametrize("name", ["dmpc_options", "dmpc_ocp_desc"])
def test_ctypes_struct_matches_header(name):
    import ctypes
    from paper_2510_06179_gb300 import _lib
    cls = getattr(_lib, name)
    fields = [f[0] for f in cls._fields_]
    c = _c_layout(name, fields)
    assert c["size"] == ctypes.sizeof(cls), (c["size"], ctypes.sizeof(cls))
    for f in fields:
        assert c[f] == getattr(cls, f).offset, (f, c[f], getattr(cls, f).offset)
