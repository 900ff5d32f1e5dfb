"""The ctypes mirrors of the C structs in include/ptycho.h have the C layout: a small C program
built with the host compiler prints sizeof and every field's offset, and the binding must agree
(a field added to the header but not to the binding, or in another order, fails here)."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "ptycho_geom_t": "Geom",
    "ptycho_adam_t": "Adam",
    "ptycho_site_t": "Site",
}
# binding field names that differ from the C names (Python keywords)
C_NAME = {"lam": "lambda"}


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    from paper_2311_14780_gb300 import _native
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ptycho.h"', "int main(void) {"]
    for cname, pyname in STRUCTS.items():
        cls = getattr(_native, pyname)
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {C_NAME.get(field, field)}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    table = {}
    for line in out:
        if line:
            s, f, v = line.split()
            table[(s, f)] = int(v)
    return table


def test_binding_structs_match_the_c_layout(tmp_path):
    from paper_2311_14780_gb300 import _native
    table = _c_layout(tmp_path)
    for cname, pyname in STRUCTS.items():
        cls = getattr(_native, pyname)
        assert ctypes.sizeof(cls) == table[(cname, "size")], cname
        for field, _ in cls._fields_:
            assert getattr(cls, field).offset == table[(cname, field)], (cname, field)


def test_header_fields_are_all_bound(tmp_path):
    """Every field of the C structs appears in the binding (checked through the sizes: a
    missing trailing field would leave the ctypes struct smaller)."""
    from paper_2311_14780_gb300 import _native
    table = _c_layout(tmp_path)
    for cname, pyname in STRUCTS.items():
        cls = getattr(_native, pyname)
        last, ftype = cls._fields_[-1]
        end = getattr(cls, last).offset + ctypes.sizeof(ftype)
        assert end <= table[(cname, "size")] < end + 8, cname


def test_binding_signatures_match_the_header_prototypes():
    """Each bound entry point takes as many arguments as its prototype in ptycho.h."""
    import re
    from paper_2311_14780_gb300 import _native
    text = open(os.path.join(ROOT, "include", "ptycho.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    protos = {}
    for m in re.finditer(r"\b(ptycho_[A-Za-z0-9_]+)\s*\(([^;{]*?)\)\s*;", text):
        name, args = m.group(1), m.group(2).strip()
        protos[name] = 0 if args in ("", "void") else len(args.split(","))
    for name, _, argtypes in _native.SIGNATURES:
        assert name in protos, name
        assert len(argtypes) == protos[name], (name, len(argtypes), protos[name])
    assert set(protos) == {n for n, _, _ in _native.SIGNATURES}      # every prototype is bound
