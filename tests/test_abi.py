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
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    assert os.path.exists(build.build())


# the binding's ctypes mirrors of the header's structs: same size, same field offsets
_STRUCTS = [("wpm_conditions", "Conditions"), ("wpm_output", "Output"),
            ("wpm_instance", "Instance"), ("wpm_tuning", "Tuning"),
            ("wpm_run_stats", "RunStats"), ("wpm_engine_config", "EngineConfig")]


def test_binding_structs_match_the_header(tmp_path):
    import subprocess
    from paper_2301_00806_gb300 import wpm
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "wpm.h"', "int main(void) {"]
    expect = {}
    for cname, pyname in _STRUCTS:
        cls = getattr(wpm, pyname)
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        expect[cname] = ctypes.sizeof(cls)
        for f, _ in cls._fields_:
            lines.append(f'  printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
            expect[f"{cname}.{f}"] = getattr(cls, f).offset
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o",
                           str(exe), str(src)])
    out = subprocess.check_output([str(exe)], text=True)
    got = {k: int(v) for k, v in (ln.split() for ln in out.split("\n") if ln.strip())}
    assert got == expect
