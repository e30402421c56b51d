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


def header_constants():
    """Every CBS_* enumerator of the header with its value."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", text, flags=re.S):
        nxt = 0
        for item in body.split(","):
            item = item.strip()
            if not item:
                continue
            m = re.match(r"(CBS_[A-Z0-9_]+)\s*(?:=\s*(-?\d+))?$", item)
            assert m, item
            nxt = int(m.group(2)) if m.group(2) is not None else nxt
            out[m.group(1)] = nxt
            nxt += 1
    return out


def test_binding_constants_match_the_header():
    consts = header_constants()
    assert len(consts) >= 20
    for name, value in consts.items():
        if hasattr(abi, name):
            assert getattr(abi, name) == value, name
    for name in ("CBS_LHS_BLOCK", "CBS_BATCH_AUTO", "CBS_BATCH_PERSISTENT", "CBS_BATCH_PER_PROBLEM",
                 "CBS_FP32_REFINE_I64", "CBS_RHS_MIDPOINT", "CBS_ERR_RANGE"):
        assert name in consts and getattr(abi, name) == consts[name], name


def _struct_fields(tag):
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (tag, tag), text, flags=re.S).group(1)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        for part in decl.split(","):
            m = re.search(r"\**\s*([a-z_0-9]+)\s*(\[\d+\])?\s*$", part.strip())
            names.append(m.group(1))
    return names


def test_struct_layouts_match_the_header():
    # field names in declaration order, against the ctypes mirrors
    assert _struct_fields("cbs_desc") == [f[0] for f in abi.cbs_desc._fields_]
    assert _struct_fields("cbs_plan_info") == [f[0] for f in abi.cbs_plan_info._fields_]


def test_struct_offsets_match_a_c_compiler(tmp_path):
    # sizeof and every field offset as gcc lays the header's structs out,
    # against the ctypes mirrors the binding passes to the library
    import shutil
    import subprocess
    import pytest
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "cbs.h"', "int main(void) {"]
    for tag, mirror in (("cbs_desc", abi.cbs_desc), ("cbs_plan_info", abi.cbs_plan_info)):
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (tag, tag))
        for name, _ in mirror._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (tag, name, tag, name))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for tag, mirror in (("cbs_desc", abi.cbs_desc), ("cbs_plan_info", abi.cbs_plan_info)):
        assert got[(tag, "sizeof")] == ctypes.sizeof(mirror), tag
        for name, _ in mirror._fields_:
            assert got[(tag, name)] == getattr(mirror, name).offset, (tag, name)
