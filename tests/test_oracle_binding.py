"""The oracle's ctypes binding against its C source: every option structure's
fields at the offsets and sizes gcc gives them, and every integer constant
(precisions, modes, patterns, stop rules, status flags) with the C value.  A
binding that drifted from the C structs would hand the oracle garbled options
without any error, so this is checked directly rather than through results."""
import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "spai_ir_oracle.c")

# C struct name -> the binding's ctypes class
STRUCTS = {"orc_spai_opts": O.SpaiOpts, "orc_gmres_opts": O.GmresOpts, "orc_ir_opts": O.IrOpts}
# C #define -> the binding's name
RENAMED = {"PH": "HALF", "PS": "SINGLE", "PD": "DOUBLE", "PQ": "QUAD"}


def c_structs():
    src = re.sub(r"/\*.*?\*/", "", open(SRC).read(), flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*([A-Za-z_]\w*)\s*;", src, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if decl:
                first, *rest = [p.strip() for p in decl.split(",")]
                fields.append(re.match(r"^.*?([A-Za-z_]\w*)$", first).group(1))
                fields += [re.match(r"^\**\s*([A-Za-z_]\w*)", p).group(1) for p in rest]
        out[name] = fields
    return out


def c_defines():
    return re.findall(r"^#define[ \t]+([A-Z][A-Z0-9_]*)[ \t]+-?\d+\b", open(SRC).read(), flags=re.M)


@pytest.fixture(scope="module")
def layout(tmp_path_factory):
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = c_structs()
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "spai_ir_oracle.c"', "int main(void) {"]
    for sname in STRUCTS:
        lines.append('    printf("%%s __size__ %%zu 0\\n", "%s", sizeof(%s));' % (sname, sname))
        for f in structs[sname]:
            lines.append('    printf("%%s %%s %%zu %%zu\\n", "%s", "%s", offsetof(%s, %s), sizeof(((%s*)0)->%s));'
                         % (sname, f, sname, f, sname, f))
    for d in c_defines():
        lines.append('    printf("#define %%s %%lld 0\\n", "%s", (long long)(%s));' % (d, d))
    lines += ["    return 0;", "}"]
    tmp = tmp_path_factory.mktemp("oracle_layout")
    src = tmp / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp / "layout"
    subprocess.run([cc, "-std=gnu11", "-fopenmp", "-I", os.path.join(ROOT, "oracle"), str(src), "-o", str(exe),
                    "-lm"], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        a, b, c, d = line.split()
        got[(a, b)] = (int(c), int(d))
    return structs, got


def test_option_structs_match_the_c_layout(layout):
    structs, got = layout
    for sname, cls in STRUCTS.items():
        assert [f for f, *_ in cls._fields_] == structs[sname], sname
        assert C.sizeof(cls) == got[(sname, "__size__")][0], sname
        for f in structs[sname]:
            d = getattr(cls, f)
            assert (d.offset, d.size) == got[(sname, f)], (sname, f)


def test_constants_match_the_c_defines(layout):
    _, got = layout
    names = [b for (a, b) in got if a == "#define"]
    assert {"PH", "MODE_ACC32", "PAT_A2", "IR_STAGNATED", "CF_NONFINITE", "STOP_CORRECTION"} <= set(names)
    for n in names:
        assert getattr(O, RENAMED.get(n, n)) == got[("#define", n)][0], n
