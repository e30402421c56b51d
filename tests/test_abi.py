"""The C-ABI library loads and exports every entry point include/cbs.h declares
(no compute calls, no GPU needed)."""
import ctypes
import os
import re

from paper_2101_02286_gb300 import abi

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "cbs.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cbs_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_entry_points():
    names = declared_functions()
    assert "cbs_plan_create" in names and "cbs_solve" in names and "cbs_batch_solve" in names
    assert set(names) == set(abi.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(abi.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_version_and_error_string():
    assert abi.cbs_version() >= 100
    assert isinstance(abi._lib.cbs_last_error_string(), bytes)
