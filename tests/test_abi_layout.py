"""CPU check that the Python binding marshals what include/gk.h declares:
every ctypes structure has the size and field offsets a C compiler gives
the header's struct, and every enum-like constant of the binding equals the
header's #define."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gk.h")

PAIRS = [("gk_criteria", "Criteria"), ("gk_status", "Status"), ("gk_solver_info", "SolverInfo"),
         ("gk_matrix_info", "MatrixInfo"), ("gk_batch_status", "BatchStatus")]


def _binding():
    import paper_2006_16852_gb300 as gk
    return gk


def _c_layout(tmp_path):
    gk = _binding()
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gk.h"', "int main(void) {"]
    for cname, pyname in PAIRS:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in getattr(gk, pyname)._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        s, f, v = line.split()
        got[(s, f)] = int(v)
    return got


def test_struct_layouts_match_the_header(tmp_path):
    gk = _binding()
    c = _c_layout(tmp_path)
    for cname, pyname in PAIRS:
        py = getattr(gk, pyname)
        assert ctypes.sizeof(py) == c[(cname, "size")], cname
        for f, _ in py._fields_:
            assert getattr(py, f).offset == c[(cname, f)], (cname, f)


def _defines():
    text = open(HEADER).read()
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(GK_\w+)\s+(-?\d+)\b", text)}


def test_constants_match_the_header():
    gk = _binding()
    d = _defines()
    fmt = {"csr": "GK_CSR", "csr_merge": "GK_CSR_MERGE", "ell": "GK_ELL", "hyb": "GK_HYB", "auto": "GK_AUTO"}
    for k, v in gk.FORMATS.items():
        assert d[fmt[k]] == v, k
    kinds = {"cg": "GK_CG", "bicgstab": "GK_BICGSTAB", "ir_cg": "GK_IR_CG", "fcg": "GK_FCG", "cgs": "GK_CGS",
             "gmres": "GK_GMRES"}
    for k, v in gk.SOLVERS.items():
        assert d[kinds[k]] == v, k
    for name in ("STOP_NONE", "STOP_CONVERGED", "STOP_MAX_ITERS", "STOP_BREAKDOWN", "STOP_NAN", "STOP_TIME",
                 "FORM_GRAPH", "FORM_HOST", "FORM_CLUSTER", "FORM_GRID"):
        assert getattr(gk, name) == d["GK_" + name], name
    assert gk.BATCH_CLASSES == d["GK_BATCH_CLASSES"]
    assert (gk.F64, gk.F32) == (d["GK_F64"], d["GK_F32"])
