"""The C-ABI library loads and exports every entry point include/spai_ir.h
declares (no compute calls: these run without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    hdr = open(os.path.join(ROOT, "include", "spai_ir.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([a-z_][a-z0-9_]*)\s*\(", hdr, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2202_10204_gb300.build import build
    return build()


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for required in ("spai_build", "gmres_ir_solve", "solver_submit", "solver_poll", "spai_ctx_create",
                     "spai_ctx_destroy", "spai_precond_free", "spai_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    out = subprocess.run(["nm", "-D", "--defined-only", built_lib], capture_output=True, text=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if " T " in line)
    missing = [n for n in declared_entry_points() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_matches(built_lib):
    import torch  # noqa: F401  (provides the CUDA runtime the library links)
    from paper_2202_10204_gb300 import _lib
    L = _lib.lib()
    for name in declared_entry_points():
        assert hasattr(L, name)
    assert set(_lib.EXPORTED) == set(declared_entry_points())
    assert _lib.strerror(-6) == "a bounded device-side wait expired"
    assert _lib.strerror(12345) == "unknown status"


def test_binding_struct_layouts_match_header():
    import ctypes as C
    from paper_2202_10204_gb300 import _lib
    # spai_csr: 2 int64 + 3 pointers + int (padded) ; ir_stats holds 64 its and 65 nbe
    assert C.sizeof(_lib.spai_csr) == 48
    assert C.sizeof(_lib.ir_stats) >= 64 * 4 + 65 * 8
    assert _lib.SPAI_IR_MAX_STEPS == int(re.search(r"#define SPAI_IR_MAX_STEPS (\d+)",
                                                   open(os.path.join(ROOT, "include", "spai_ir.h")).read()).group(1))


def header_structs():
    """{struct name: [field names in order]} of every typedef'd struct in the header."""
    hdr = open(os.path.join(ROOT, "include", "spai_ir.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*([A-Za-z_]\w*)\s*;", hdr, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            first, *rest = [p.strip() for p in decl.split(",")]
            fields.append(re.match(r"^.*?([A-Za-z_]\w*)\s*(\[[^\]]*\])?$", first).group(1))
            fields += [re.match(r"^\**\s*([A-Za-z_]\w*)", p).group(1) for p in rest]
        out[name] = fields
    return out


def test_binding_field_offsets_match_the_c_compiler(tmp_path):
    # every field of every struct the header declares, at the offset and size the
    # C compiler gives it, in the ctypes structure the binding passes across the ABI
    import ctypes as C
    import shutil
    from paper_2202_10204_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = header_structs()
    assert set(structs) >= {"spai_csr", "spai_opts", "ir_opts", "spai_stats", "ir_stats"}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "spai_ir.h"', "int main(void) {"]
    for sname, fields in structs.items():
        lines.append('    printf("%%s __size__ %%zu 0\\n", "%s", sizeof(%s));' % (sname, sname))
        for f in fields:
            lines.append('    printf("%%s %%s %%zu %%zu\\n", "%s", "%s", offsetof(%s, %s), sizeof(((%s*)0)->%s));'
                         % (sname, f, sname, f, sname, f))
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        sname, f, off, size = line.split()
        got[(sname, f)] = (int(off), int(size))
    for sname, fields in structs.items():
        cls = getattr(_lib, sname)
        assert [f for f, *_ in cls._fields_] == fields, sname
        assert C.sizeof(cls) == got[(sname, "__size__")][0], sname
        for f in fields:
            d = getattr(cls, f)
            assert (d.offset, d.size) == got[(sname, f)], (sname, f)


def header_constants():
    """Names of the header's integer constants: its #defines and enumerators."""
    hdr = open(os.path.join(ROOT, "include", "spai_ir.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    defines = re.findall(r"^#define[ \t]+([A-Z][A-Z0-9_]*)[ \t]+\S", hdr, flags=re.M)
    enums = [n for body in re.findall(r"typedef enum\s*\{(.*?)\}", hdr, flags=re.S)
             for n in re.findall(r"([A-Z][A-Z0-9_]*)\s*=", body)]
    return defines + enums


def test_binding_constants_match_the_header(tmp_path):
    # every status code, precision, pattern and stop-rule value the header defines has the
    # same value under its binding name (SPAI_ prefix dropped, except SPAI_IR_MAX_STEPS)
    import shutil
    from paper_2202_10204_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = header_constants()
    assert "SPAI_ERR_TIMEOUT" in names and "SPAI_HALF" in names and "IR_STOP_CORRECTION" in names
    lines = ["#include <stdio.h>", '#include "spai_ir.h"', "int main(void) {"]
    lines += ['    printf("%%s %%lld\\n", "%s", (long long)(%s));' % (n, n) for n in names]
    lines += ["    return 0;", "}"]
    src = tmp_path / "consts.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "consts"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    values = dict((n, int(v)) for n, v in (line.split() for line in subprocess.run(
        [str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()))
    no_binding = {"SPAI_NOALLOC_SCRATCH_BYTES"}  # a size, documented in the header only
    for n, v in values.items():
        if n in no_binding:
            continue
        py = n if n == "SPAI_IR_MAX_STEPS" or not n.startswith("SPAI_") else n[len("SPAI_"):]
        assert getattr(_lib, py) == v, n


def test_package_exports_every_status_code_and_entry_point():
    import paper_2202_10204_gb300 as S
    from paper_2202_10204_gb300 import _lib
    codes = [n for n in header_constants() if n.startswith(("SPAI_ERR_", "SPAI_WARN_")) or n in ("SPAI_OK",
                                                                                                "SPAI_PENDING")]
    for n in codes:
        assert getattr(S, n[len("SPAI_"):]) == getattr(_lib, n[len("SPAI_"):]), n
    for name in ("gmres_ir_solve", "gmres_ir_solve_batch", "gmres_ir_solve_noalloc", "spai_build",
                 "spai_build_batch", "solver_submit", "solver_poll", "strerror", "tune_get", "tune_set",
                 "selftest_wait_timeout", "Context", "Precond"):
        assert getattr(S, name) is getattr(_lib, name), name
    assert set(S.__all__) <= set(dir(S))


def test_argument_checks_return_before_any_device_work(built_lib):
    # NULL handles and out-of-range options are refused with SPAI_ERR_INVALID_ARG before any
    # CUDA call (so these run without a GPU); the tuner's table is host state
    import torch  # noqa: F401  (provides the CUDA runtime the library links)
    from paper_2202_10204_gb300 import _lib
    L, E = _lib.lib(), _lib.ERR_INVALID_ARG
    assert L.spai_ctx_create(None, 0, None, 0) == E
    assert L.spai_build(None, None, None, None, None) == E
    assert L.spai_build_batch(None, 0, None, None, None, None, None) == E
    assert L.gmres_ir_solve(None, None, None, None, None, None, None, None) == E
    assert L.gmres_ir_solve_batch(None, 0, None, None, None, None, None, None, None) == E
    assert L.gmres_ir_solve_noalloc(None, None, None, None, None, None, None) == E
    assert L.solver_submit(None, None, None, None, None, None) == E
    assert L.solver_poll(None, 0, None, None) == E
    assert L.spai_precond_info(None, None, None) == E
    assert L.spai_precond_export(None, None, None, None) == E
    for mode, limit in ((2, 50.0), (0, 0.0), (0, -1.0), (0, 2e4)):
        assert L.spai_selftest_wait_timeout(0, mode, limit) == E
    L.spai_ctx_destroy(None)
    L.spai_precond_free(None)
    for bad in ((0, 1, 1), (0, 1, 14), (0, 7, 5), (0, _lib.QUAD, 5)):
        assert L.spai_tune_get(*bad) == E
        assert L.spai_tune_set(*bad, 0) == E
    assert L.spai_tune_set(0, _lib.SINGLE, 5, 4) == E and L.spai_tune_set(0, _lib.SINGLE, 5, -2) == E
    dev = 97  # a device index no test builds on
    assert L.spai_tune_get(dev, _lib.HALF, 5) == -1
    assert L.spai_tune_set(dev, _lib.HALF, 5, 2) == 0 and L.spai_tune_get(dev, _lib.HALF, 5) == 2
    assert L.spai_tune_get(dev, _lib.SINGLE, 5) == -1 and L.spai_tune_get(dev, _lib.HALF, 6) == -1
    assert L.spai_tune_set(dev, _lib.HALF, 5, -1) == 0 and L.spai_tune_get(dev, _lib.HALF, 5) == -1


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # no CPU fallback: without the built library every entry point raises
    from paper_2202_10204_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "absent" / "libspai_ir.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.lib()
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.Context(0)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.strerror(0)


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2202_10204_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src and "spai_ir_oracle" not in src, f


def test_strerror_names_every_code():
    import paper_2202_10204_gb300 as S
    from paper_2202_10204_gb300 import _lib
    codes = [0, 1, 2, 3] + [-i for i in range(1, 11)]
    names = [S.strerror(c) for c in codes]
    assert all(isinstance(n, str) and n and n != "unknown status" for n in names)
    assert len(set(names)) == len(names)
    assert S.strerror(-99) == "unknown status"
