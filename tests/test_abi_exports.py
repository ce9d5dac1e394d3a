"""The C-ABI library loads and exports every function include/pm4g.h declares
(no GPU needed: nothing is called)."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pm4g.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pm4g_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2204_04898_b300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared()
    for must in ("pm4g_load_log", "pm4g_dfg", "pm4g_perf_dfg", "pm4g_start_end", "pm4g_variants",
                 "pm4g_filter", "pm4g_filter_paths", "pm4g_filter_cases", "pm4g_efg", "pm4g_log_free",
                 "pm4g_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (pm4g_\w+)", out))
    assert set(declared()) <= exported


def test_binding_names_match_the_abi():
    from paper_2204_04898_b300 import pm4g
    for n in declared():
        if n.endswith("_free") and n not in ("pm4g_log_free",):
            continue  # result frees are called inside the binding
        assert hasattr(pm4g, n), n


def test_binding_loads_without_gpu():
    from paper_2204_04898_b300 import pm4g
    assert "segment" in pm4g.pm4g_kernel_names()
