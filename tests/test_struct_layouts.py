"""The ctypes structures of the binding have the C layout of include/hodlr_mf.h: a small
C program compiled against the header prints sizeof and the offset of every field the
binding declares, and they must equal the ctypes figures (a field added on one side
only would shift every later field).  Host compiler only; no GPU."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PAIRS = [("hm_opts", "HmOpts"), ("hm_solve_info", "HmSolveInfo"), ("hm_factor_info", "HmFactorInfo"),
         ("hm_server_stats", "HmServerStats"), ("hm_prof_entry", "HmProfEntry")]


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no host C compiler")
def test_binding_structs_match_the_header(tmp_path):
    import paper_1410_2697_gb300._binding as b
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "hodlr_mf.h"', "int main(void) {"]
    expect = []
    for cname, pyname in PAIRS:
        cls = getattr(b, pyname)
        lines.append(f'  printf("%zu\\n", sizeof({cname}));')
        expect.append(ctypes.sizeof(cls))
        for field, _ in cls._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {field}));')
            expect.append(getattr(cls, field).offset)
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == expect
