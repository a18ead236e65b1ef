"""The C-ABI library loads and exports every entry point include/pdw1.h
declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pdw1.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pd_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("pd_condense", "pd_rwmd_lower_bound", "pd_wspd_sparsify", "pd_w1_approx", "pd_mcf_solve",
                 "pd_create", "pd_destroy", "pd_last_error", "pd_opts_default"):
        assert must in names


def test_library_builds_and_exports_every_symbol():
    from paper_2110_14734_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_struct_layouts_match_header():
    """ctypes mirrors of the structs have the header's field order."""
    from paper_2110_14734_gb300 import build
    build.build()
    from paper_2110_14734_gb300 import pdw1
    src = open(os.path.join(ROOT, "include", "pdw1.h")).read()
    body = re.search(r"typedef struct \{((?:(?!typedef struct).)*?)\} pd_result;", src, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"(\w+)(?:\[\d+\])?\s*;", body)
    assert fields == [f for f, _ in pdw1.pd_result._fields_]
    body = re.search(r"typedef struct \{((?:(?!typedef struct).)*?)\} pd_opts;", src, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"(\w+)\s*;", body)
    assert fields == [f for f, _ in pdw1.pd_opts._fields_]
