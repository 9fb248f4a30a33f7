"""The C-ABI library builds, loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hodlr_mf.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hm_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__
    return __graft_entry__._builder().build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["hm_create", "hm_analyze", "hm_factor", "hm_solve", "hm_destroy",
                     "hm_ctx_destroy", "hm_status_str", "hm_get_ordering", "hm_precond_apply"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (hm_[a-z_]+)$", out, flags=re.M))
    assert set(declared_functions()) <= exported


def test_binding_mirrors_header(lib_path):
    import paper_1410_2697_gb300._binding as b
    assert set(b.EXPORTED) == set(declared_functions())
    for name in b.EXPORTED:
        if name not in ("hm_status_str", "hm_last_error"):
            assert callable(getattr(b, name))
        # every entry point has its C argument types (ctypes cannot pass a float without them)
        assert getattr(b._lib, name).argtypes is not None, name


def test_status_strings_without_gpu(lib_path):
    import paper_1410_2697_gb300._binding as b
    assert b.hm_status_str(0) == "ok"
    assert "converge" in b.hm_status_str(3)
    o = b.hm_default_opts()
    assert (o.nd_leaf, o.hodlr_leaf, o.n_c, o.restart) == (64, 64, 64, 30)


def test_oracle_is_not_imported_by_the_product():
    pkg = os.path.join(ROOT, "paper_1410_2697_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.findall(r"^\s*(?:from|import)\s+(\w+)", txt, flags=re.M), f
