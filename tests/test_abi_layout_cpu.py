"""The ctypes binding's structures against include/tm.h as a C compiler lays
them out: for every `typedef struct { ... } name;` of the header, the binding's
class of the same name has the same members in the same order, at the same
offsets, with the same total size.  A drift here (a member added to the header
but not to the binding) would shift every later field of the call."""
import ctypes as ct
import pathlib
import re
import shutil
import subprocess

import pytest

ROOT = pathlib.Path(__file__).resolve().parents[1]
HDR = ROOT / "include" / "tm.h"


def _structs():
    text = re.sub(r"/\*.*?\*/", "", HDR.read_text(), flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*(\w+)\s*;", text, flags=re.S):
        members = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            m = re.match(r"([\w\s]+?)\s+(\w.*)$", decl)
            for part in m.group(2).split(","):
                members.append(re.match(r"\s*(\w+)", part).group(1))
        out[name] = members
    return out


def test_header_structs_are_found():
    s = _structs()
    assert {"tm_params", "tm_solve_params", "tm_solve_info", "tm_mg_params", "tm_tuning"} <= set(s)


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_binding_structs_match_the_c_layout(tmp_path):
    from paper_2212_06635_gb300 import tm
    structs = _structs()
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HDR}"', "int main(void) {"]
    for name, members in structs.items():
        lines.append(f'    printf("%s size %zu\\n", "{name}", sizeof({name}));')
        for mem in members:
            lines.append(f'    printf("%s %s %zu\\n", "{name}", "{mem}", offsetof({name}, {mem}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", str(src), "-o", str(exe)], check=True)
    c_layout = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        name, key, val = line.split()
        c_layout[(name, key)] = int(val)
    for name, members in structs.items():
        cls = getattr(tm, name)
        assert [f for f, _ in cls._fields_] == members, name
        assert ct.sizeof(cls) == c_layout[(name, "size")], name
        for mem in members:
            assert getattr(cls, mem).offset == c_layout[(name, mem)], (name, mem)


def _prototypes():
    text = re.sub(r"/\*.*?\*/", "", HDR.read_text(), flags=re.S)
    out = {}
    for ret, name, args in re.findall(r"(tm_status|const char\s*\*)\s+(tm_\w+)\s*\(([^)]*)\)\s*;", text):
        out[name] = [a.strip() for a in args.split(",")] if args.strip() not in ("", "void") else []
    return out


def _c_kind(decl):
    if "*" in decl or "[" in decl:
        return "p"
    t = decl.rsplit(None, 1)[0] if len(decl.split()) > 1 else decl
    if "double" in t:
        return "d"
    if "long long" in t:
        return "q"
    return "i"   # int and the tm_* enums


def _ct_kind(t):
    if t in (ct.c_void_p, ct.c_char_p) or hasattr(t, "_type_") and isinstance(t, type) and issubclass(t, ct._Pointer):
        return "p"
    return {ct.c_double: "d", ct.c_int: "i", ct.c_ulonglong: "q"}[t]


def test_binding_signatures_match_the_header():
    """Every bound entry point takes the header's number and kinds of arguments
    (pointer, int or enum, double, 64-bit integer), in order."""
    from paper_2212_06635_gb300 import tm
    protos = _prototypes()
    assert len(protos) >= 50
    for name, argtypes in tm._sigs.items():
        assert name in protos, name
        c_kinds = [_c_kind(a) for a in protos[name]]
        py_kinds = [_ct_kind(t) for t in argtypes]
        assert c_kinds == py_kinds, (name, c_kinds, py_kinds)
