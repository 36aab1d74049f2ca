"""The ctypes mirror of exa_result matches the C struct of include/exa.h field by field (size
and offsets), checked by compiling a small C program against the header (CPU only)."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FIELDS = ["loglik", "logdet", "quad", "ir_resid", "ir_iters", "tile_nb", "exact_band", "n_tiles", "ms_gen", "ms_chol",
          "ms_solve", "ms_total", "quad_err"]


def test_exa_result_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1908_06936_gb300 import ExaResult

    src = tmp_path / "layout.c"
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "exa.h"', "int main(void) {",
             '  printf("size %zu\\n", sizeof(exa_result));']
    for f in FIELDS:
        lines.append('  printf("%s %%zu\\n", offsetof(exa_result, %s));' % (f, f))
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                   text=True).stdout.splitlines())
    assert int(out["size"]) == ctypes.sizeof(ExaResult)
    assert [f for f, _ in ExaResult._fields_] == FIELDS
    for f in FIELDS:
        assert int(out[f]) == getattr(ExaResult, f).offset, f
