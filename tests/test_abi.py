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
