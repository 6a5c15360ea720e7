"""The C-ABI library builds, loads and exports every entry point that
include/pdfgb.h declares; the ctypes structs match the C layout.  No GPU
work is done here."""
import os
import re
import subprocess
import ctypes

import pytest

import paper_1006_0720_gb300 as pg
from paper_1006_0720_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pdfgb.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pdf_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for need in ("pdf_mesh_create", "pdf_particles_init", "pdf_step", "pdf_estimate_stats"):
        assert need in names


def test_library_exports_every_declared_symbol():
    L = pg.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
        assert name in capi.PROTOTYPES, "binding lacks " + name


def test_every_exported_entry_point_is_declared_and_documented():
    """The reverse direction: each pdf_* symbol the library exports is
    declared in the header and preceded there by a comment block."""
    so = pg.lib()._name
    out = subprocess.check_output(["nm", "-D", "--defined-only", so]).decode()
    exported = sorted({ln.split()[-1] for ln in out.splitlines() if re.search(r" T pdf_[a-z0-9_]+$", ln)})
    assert len(exported) > 20
    declared = set(declared_functions())
    text = open(HEADER).read()
    for name in exported:
        assert name in declared, "undeclared export " + name
        # the declaration: a line that starts with its return type
        m = re.search(r"^[A-Za-z_][\w \t\*]*\b" + name + r"\s*\(", text, flags=re.M)
        assert m, name
        before = text[:m.start()].rstrip()
        # it follows a comment, directly or after other declarations of its group
        assert "*/" in before[max(0, len(before) - 3000):], name


def test_struct_layouts_match_the_header(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "%s"\n'
                   'int main(void){printf("%%zu %%zu %%zu %%zu %%zu\\n", sizeof(pdf_model_params),'
                   ' sizeof(pdf_init_params), sizeof(pdf_step_info), offsetof(pdf_model_params, C1),'
                   ' offsetof(pdf_init_params, u_sigma)); return 0;}\n' % HEADER)
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-std=c11", "-o", str(exe), str(src)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert got == [ctypes.sizeof(capi.ModelParams), ctypes.sizeof(capi.InitParams),
                   ctypes.sizeof(capi.StepInfo), capi.ModelParams.C1.offset,
                   capi.InitParams.u_sigma.offset]


def test_default_parameters_are_the_papers_constants():
    p = pg.model_params()
    golden = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "model_constants.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            golden[k] = float(v)
    for k, v in golden.items():
        assert getattr(p, k) == v, k
    # micromixing constants of the concentrated-source form (table of constants, ch. 5)
    assert p.Cs == 0.02 and p.Ct == 0.7


def test_errors_are_reported_not_raised_in_c():
    L = pg.lib()
    st = L.pdf_mesh_create(None, 0, None, 0, None, None, 0, 0.0, None)
    assert st == capi.PDF_EINVAL
    assert "out is NULL" in pg.pdf_last_error()
