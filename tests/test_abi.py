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


def test_binding_struct_offsets_match_the_c_compiler(tmp_path):
    """Every field of every public struct sits at the offset, and every struct
    has the size, that a C compiler gives it from include/pdw1.h."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2110_14734_gb300 import build
    build.build()
    from paper_2110_14734_gb300 import pdw1
    structs = {"pd_diagram": pdw1.pd_diagram, "pd_opts": pdw1.pd_opts, "pd_nodes": pdw1.pd_nodes,
               "pd_network": pdw1.pd_network, "pd_result": pdw1.pd_result, "pd_nn_result": pdw1.pd_nn_result,
               "pd_ws_stats": pdw1.pd_ws_stats}
    lines = ['#include "pdw1.h"', "#include <stddef.h>", "#include <stdio.h>", "int main(void) {"]
    for name, cls in structs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for f, _ in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            k, v = line.rsplit(" ", 1)
            got[k] = int(v)
    for name, cls in structs.items():
        assert got["%s size" % name] == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got["%s %s" % (name, f)] == getattr(cls, f).offset, (name, f)
