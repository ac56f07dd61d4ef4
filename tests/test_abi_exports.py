"""The C-ABI library builds, loads and exports every function include/dbscan.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1506_02226_gb300 import binding
from paper_1506_02226_gb300 import build as build_mod

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "dbscan.h")


def _declared_functions():
    with open(HEADER) as f:
        txt = f.read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(dbscan_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    return build_mod.build()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("dbscan_plan_create", "dbscan_plan_destroy", "dbscan_run", "dbscan_batch",
                 "dbscan_serve_submit", "dbscan_strerror"):
        assert must in names


def test_every_declared_symbol_is_exported(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (\w+)", out))
    missing = [n for n in _declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_covers_the_header(libpath):
    assert sorted(binding.exported_symbols()) == _declared_functions()
    L = binding.lib()
    for n in _declared_functions():
        assert isinstance(getattr(L, n), ctypes._CFuncPtr)


def test_host_only_calls(libpath):
    assert binding.dbscan_abi_version() == 2
    assert binding.dbscan_strerror(binding.DBSCAN_ERR_NOT_QUANTISED).startswith("a coordinate")
    assert binding.dbscan_strerror(12345) == "unknown status"
    o = binding.dbscan_opts_default()
    assert (o.max_d, o.synchronous, o.grid, o.label_mode) == (64, 1, 0, 0)
    s = binding.dbscan_serve_opts_default()
    assert s.slots >= 1 and s.hbm_budget_bytes == 120 << 30


def test_struct_layouts_match_header():
    assert ctypes.sizeof(binding.dbscan_opts) == 72
    assert ctypes.sizeof(binding.dbscan_stats) == 96
    assert ctypes.sizeof(binding.dbscan_instance) == 40
    assert binding.dbscan_instance.labels_out.offset == 32
    assert binding.dbscan_stats.pair_tests.offset == 72


def test_header_is_plain_c(tmp_path):
    """The boundary is usable from C: the header compiles as C11 with warnings
    as errors (pedantic), and its struct sizes are the ones the binding marshals."""
    import shutil
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi_check.c"
    src.write_text(
        '#include "dbscan.h"\n'
        "_Static_assert(sizeof(dbscan_opts) == 72, \"opts\");\n"
        "_Static_assert(sizeof(dbscan_stats) == 96, \"stats\");\n"
        "_Static_assert(sizeof(dbscan_instance) == 40, \"instance\");\n"
        "_Static_assert(offsetof(dbscan_stats, pair_tests) == 72, \"stats.pair_tests\");\n"
        "int use(dbscan_plan *p, const float *x, int32_t *l) {\n"
        "    dbscan_opts o; dbscan_opts_default(&o);\n"
        "    return dbscan_run(p, x, 0, 2, 0.1f, 5, l, (dbscan_stats *)0);\n"
        "}\n")
    inc = os.path.join(os.path.dirname(__file__), "..", "include")
    r = subprocess.run(["gcc", "-std=c11", "-pedantic", "-Wall", "-Wextra", "-Werror", "-fsyntax-only", "-I", inc, str(src)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
