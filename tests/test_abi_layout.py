"""The ctypes binding agrees with include/wsm.h: every prototype's return and
parameter kinds, the layout of every struct the binding mirrors (offsets and
sizes as a C compiler lays them out on this machine), and the constants
(error codes, stage bits, palette and pixel limits).  No GPU, no library
load: the header is compiled with the host C compiler."""
import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

from paper_1011_0093_gb300 import _native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wsm.h")


def _header_text():
    with open(HEADER) as f:
        text = f.read()
    return re.sub(r"/\*.*?\*/", " ", text, flags=re.S)    # drop comments


def prototypes():
    """{name: (return type, [parameter types])} of every WSM_API function."""
    out = {}
    for m in re.finditer(r"WSM_API\s+([^;{]*?)\b(wsm_\w+)\s*\(([^)]*)\)\s*;", _header_text()):
        ret, name, params = m.group(1).strip(), m.group(2), m.group(3).strip()
        types = []
        if params not in ("", "void"):
            for p in params.split(","):
                p = " ".join(p.split())
                pm = re.match(r"(.*?)(\w+)$", p)   # drop the parameter name
                types.append(pm.group(1).strip())
        out[name] = (ret, types)
    return out


def kind_of_c(t):
    t = t.replace("const ", "").strip()
    if "*" in t or t == "wsm_stream":
        return "ptr"
    return {"int": "i32", "int64_t": "i64", "uint64_t": "u64", "double": "f64",
            "unsigned": "u32", "unsigned int": "u32", "uint32_t": "u32"}[t]


def kind_of_ctypes(t):
    if t in (C.c_void_p, C.c_char_p) or (isinstance(t, type) and issubclass(t, C._Pointer)):
        return "ptr"
    return {C.c_int: "i32", C.c_int64: "i64", C.c_uint64: "u64", C.c_double: "f64",
            C.c_uint: "u32"}[t]


def test_every_prototype_matches_the_binding():
    protos = prototypes()
    assert len(protos) == len(N.SIGNATURES) >= 30
    for name, (ret, params) in protos.items():
        res, args = N.SIGNATURES[name]
        assert kind_of_c(ret) == kind_of_ctypes(res), f"{name}: returns {ret}"
        assert len(params) == len(args), f"{name}: {len(params)} parameters, binding {len(args)}"
        for q, (p, a) in enumerate(zip(params, args)):
            assert kind_of_c(p) == kind_of_ctypes(a), f"{name} parameter {q}: {p} vs {a}"


STRUCTS = [("wsm_item", N.WsmItem), ("wsm_server_config", N.ServerConfig),
           ("wsm_request", N.Request), ("wsm_result", N.Result),
           ("wsm_server_stats", N.ServerStats)]


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs a C compiler")
def test_struct_layouts_match_the_c_compiler(tmp_path):
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "wsm.h"', 'int main(void) {']
    for cname, py in STRUCTS:
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["return 0;", "}"]
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.dirname(HEADER),
                    str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True,
                               text=True).stdout.splitlines():
        s, f, v = line.split()
        got[(s, f)] = int(v)
    for cname, py in STRUCTS:
        assert got[(cname, "sizeof")] == C.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, f"{cname}.{field}"


def test_header_structs_have_no_fields_the_binding_lacks():
    text = _header_text()
    for cname, py in STRUCTS:
        body = re.search(r"typedef struct\s*\{([^}]*)\}\s*" + cname + r"\s*;", text).group(1)
        names = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            first, *rest = decl.split(",")
            names.append(re.match(r".*?(\w+)$", first).group(1))
            names += [r.strip() for r in rest]
        assert names == [f for f, _ in py._fields_], cname


def _header_constants():
    vals = {}
    for m in re.finditer(r"\b(WSM_\w+)\s*=\s*(-?\d+)", _header_text()):
        vals[m.group(1)] = int(m.group(2))
    for m in re.finditer(r"#define\s+(WSM_\w+)\s+\(?(\d+)(?:ll)?\s*(?:<<\s*(\d+))?\)?",
                         _header_text()):
        vals[m.group(1)] = int(m.group(2)) << int(m.group(3) or 0)
    return vals


def test_constants_match_the_header():
    v = _header_constants()
    assert v["WSM_OK"] == N.WSM_OK
    for code, name in N.ERRORS.items():
        assert v[name] == code, name
    assert v["WSM_MAX_K"] == N.MAX_K and v["WSM_MAX_K_WIDE"] == N.MAX_K_WIDE
    assert v["WSM_MAX_PIXELS"] == N.MAX_PIXELS
    stages = {k: val for k, val in v.items() if k.startswith("WSM_STAGE_")}
    assert len(stages) == 7
    for k, val in stages.items():
        assert getattr(N, k[len("WSM_"):]) == val, k
    bits = [val for k, val in stages.items() if k != "WSM_STAGE_ALL"]
    assert sum(bits) == stages["WSM_STAGE_ALL"] and all(b & (b - 1) == 0 for b in bits)
