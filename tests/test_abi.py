"""The C ABI library builds for sm_103a, loads without a GPU, and exports every function
that include/wpm.h declares. No compute call is made here."""
import ctypes
import os
import re

from paper_2301_00806_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(wpm_\w+)\s*\(", text, re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for want in ("wpm_candidate_facets", "wpm_enumerate", "wpm_enumerate_facets",
                 "wpm_enumerate_batch", "wpm_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(build.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_library_is_built_for_sm_103a():
    path = build.build()
    data = open(path, "rb").read()
    assert b"sm_103a" in data or b"sm_103" in data
