"""The ctypes mirrors of the structs include/exa.h passes across the boundary (exa_result,
exa_kernel_stat, exa_timeline_rec) match the C structs field by field: names and order from the
header's own definition, size and offsets from a small C program compiled against it (CPU only)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_struct_fields(name):
    src = open(os.path.join(ROOT, "include", "exa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + r"\s*;", src).group(1)
    return re.findall(r"\b(\w+)\s*(?:\[\d+\])?\s*;", body)


def _mirror(name):
    import paper_1908_06936_gb300 as exa

    return {"exa_result": exa.ExaResult, "exa_kernel_stat": exa.KernelStat, "exa_timeline_rec": exa.TimelineRec}[name]


@pytest.mark.parametrize("name", ["exa_result", "exa_kernel_stat", "exa_timeline_rec"])
def test_struct_layout(tmp_path, name):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirror = _mirror(name)
    fields = header_struct_fields(name)
    assert [f for f, _ in mirror._fields_] == fields
    src = tmp_path / "layout.c"
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "exa.h"', "int main(void) {",
             '  printf("size %%zu\\n", sizeof(%s));' % name]
    for f in fields:
        lines.append('  printf("%s %%zu\\n", offsetof(%s, %s));' % (f, name, f))
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                   text=True).stdout.splitlines())
    assert int(out["size"]) == ctypes.sizeof(mirror)
    for f in fields:
        assert int(out[f]) == getattr(mirror, f).offset, f
