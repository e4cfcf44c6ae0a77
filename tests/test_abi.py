"""The C-ABI library loads on a machine without a GPU and exports every entry
point that include/wilson_mg.h declares (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1005_3043_gb300 as wmg
from paper_1005_3043_gb300 import build as wbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))]


def declared_functions():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?(?:int|void|char|double)\s*\**\s*(mg_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    wbuild.build()
    return wmg.load()


def test_header_declares_entry_points():
    names = declared_functions()
    assert {"mg_create", "mg_destroy", "mg_set_links", "mg_set_mass", "mg_setup", "mg_solve"} <= names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", wbuild.LIB], capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = declared_functions() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    for name in declared_functions():
        assert hasattr(lib, name)


def test_binding_covers_every_declared_symbol():
    assert declared_functions() <= set(wmg.EXPORTED)


def test_host_only_calls(lib):
    p = wmg.mg_default_params()
    assert p.nvec == 8 and tuple(p.block) == (4, 4, 4, 4) and p.omega == 0.9 and p.tol == 1e-10
    assert wmg.status_string(0) == "MG_OK"
    assert wmg.status_string(wmg.MG_ERR_NUMERIC) == "MG_ERR_NUMERIC"


@pytest.mark.parametrize("cname,pytype", [("mg_params", wmg.MgParams), ("mg_solve_info", wmg.MgSolveInfo)])
def test_struct_matches_header(cname, pytype):
    """The binding's structs have the header's fields, in order and with the
    same C types (int / double / int[4])."""
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "wilson_mg.h")).read(), flags=re.S)
    body = re.search(r"typedef\s+struct\s*\{([^{}]*)\}\s*" + cname + r"\s*;", src).group(1)
    fields = []
    for decl in body.split(";"):
        m = re.match(r"\s*(int|double)\s+(\w+)\s*(\[\s*(\d+)\s*\])?\s*$", decl)
        if m:
            fields.append((m.group(2), m.group(1), int(m.group(4)) if m.group(4) else None))
    assert fields, "no fields parsed"
    ct = {"int": ctypes.c_int, "double": ctypes.c_double}
    got = [(n, t) for n, t in pytype._fields_]
    assert [f[0] for f in fields] == [n for n, _ in got]
    for (name, ctype, arr), (_, t) in zip(fields, got):
        want = ct[ctype] * arr if arr else ct[ctype]
        assert t == want or (arr and t._type_ is ct[ctype] and t._length_ == arr), name
