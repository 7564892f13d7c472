"""The Python binding's ctypes mirrors of the structs that include/sfci.h
declares (sfci_params, sfci_step_info) have the C layout: the same size, and
each field at the same offset with the same size.  A field added on one side
only, or in a different order, would make every later field read garbage.
The ground truth is a small C program compiled against the header with the
host compiler; no GPU is needed."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from conftest import ROOT


def _c_layout(tmp_path, structs):
    """{struct: (sizeof, {field: (offset, size)})} from the C compiler."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "sfci.h"', "int main(void) {"]
    for cname, fields in structs.items():
        lines.append(f'    printf("S {cname} %zu\\n", sizeof({cname}));')
        for f in fields:
            lines.append(f'    printf("F {cname} {f} %zu %zu\\n", offsetof({cname}, {f}), '
                         f"sizeof((({cname} *)0)->{f}));")
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        parts = line.split()
        if parts[0] == "S":
            layout.setdefault(parts[1], [0, {}])[0] = int(parts[2])
        else:
            layout.setdefault(parts[1], [0, {}])[1][parts[2]] = (int(parts[3]), int(parts[4]))
    return layout


def test_binding_structs_match_header(tmp_path):
    import paper_2312_01846_gb300 as sf
    mirrors = {"sfci_params": sf.Params, "sfci_step_info": sf.StepInfo}
    layout = _c_layout(tmp_path, {c: [f for f, _ in py._fields_] for c, py in mirrors.items()})
    for cname, py in mirrors.items():
        size, fields = layout[cname]
        assert C.sizeof(py) == size, (cname, C.sizeof(py), size)
        for f, _ in py._fields_:
            d = getattr(py, f)
            assert (d.offset, d.size) == fields[f], (cname, f, (d.offset, d.size), fields[f])
