"""The C-ABI library loads on a machine without a GPU and exports every entry point that
include/tnsa.h declares (no compute calls are made here)."""
import ctypes
import os
import re

from paper_2507_20667_gb300 import tnsa

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "tnsa.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tn_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for core in ("tn_build", "tn_plan_create", "tn_plan_counts", "tn_plan_export", "tn_ctx_create",
                 "tn_contract", "tn_permute", "tn_program_run"):
        assert core in names


def test_every_declared_symbol_is_exported():
    lib = ctypes.CDLL(tnsa.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    assert set(declared_functions()) <= set(tnsa._SIGS)


def test_status_strings_and_version():
    assert tnsa.lib.tn_status_str(tnsa.TN_EBUDGET).decode() == "device memory budget exceeded"
    assert "sm_103a" in tnsa.tn_version()
