"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol.

No GPU needed: only calls that touch no CUDA API are made.
"""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def declared_functions():
    text = open(os.path.join(ROOT, "include", "tc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*([a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("tc_build_csr", "tc_count", "tc_edge_support", "ktruss", "ktruss_max",
              "tc_num_edges", "tc_edges", "tc_graph_free", "tc_strerror"):
        assert n in names


def test_library_builds_and_exports_every_symbol():
    import paper_1708_06866_gb300 as tc
    path = tc._build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_and_hooks_without_gpu():
    import paper_1708_06866_gb300 as tc
    assert tc.tc_strerror(0) == "ok"
    assert tc.tc_strerror(tc.TC_ERANGE) == "vertex id out of range"
    assert tc.tc_strerror(12345) == "unknown error"
    prev = tc.tc_debug_fail_alloc(3)
    assert tc.tc_debug_fail_alloc(prev) == 3
    old = tc.tc_debug_spin_limit_ns(123456)
    assert tc.tc_debug_spin_limit_ns(old) == 123456


def test_library_is_sm103a_only():
    import paper_1708_06866_gb300 as tc
    assert "arch=compute_103a,code=sm_103a" in tc._build.ARCH
    assert len(tc._build.ARCH) == 2


def test_product_package_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1708_06866_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.lower().replace("oracles", ""), f
