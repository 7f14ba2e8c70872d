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
