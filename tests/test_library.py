"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/mhar.h declares.  Host-only calls; no GPU needed."""
import os
import re

import pytest

from paper_2104_07097_gb300 import build as libbuild
from paper_2104_07097_gb300 import mhar

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(mhar_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return mhar.load()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert {"mhar_create", "mhar_run", "mhar_destroy"} <= declared
    for name in declared:
        assert hasattr(lib, name), name


def test_binding_covers_header(lib):
    assert _declared() <= set(mhar.EXPORTS)


def test_host_only_calls(lib):
    o = mhar.mhar_default_opts()
    assert o.precision == mhar.FP64 and o.refresh_k == 64 and o.graph_chunk == 16
    assert o.seed == 0 and o.walker0 == 0 and o.out_on_device == 0
    assert mhar.mhar_strerror(mhar.E_UNBOUNDED) == "MHAR_E_UNBOUNDED"
    assert mhar.mhar_strerror(12345) == "MHAR_E_UNKNOWN"


def test_struct_layout_matches_header(lib, tmp_path):
    """The ctypes mirrors have the sizes and field offsets a C compiler gives
    the header's structs (compiled here with gcc, host only)."""
    import ctypes
    import subprocess
    fields = {"mhar_opts": mhar.MharOpts, "mhar_stats": mhar.MharStats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "mhar.h"', "int main(void) {"]
    for cname, py in fields.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        cname, what, val = line.split()
        got[(cname, what)] = int(val)
    for cname, py in fields.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_status_code_mapping(lib):
    """mhar_run's return code for a device status word (no GPU needed): a
    bounded wait that ran out wins, then non-finite values, then a refresh
    beyond the tracked slack's bound, then an open chord; stalls alone are
    fine."""
    assert mhar.mhar_status_code(0, 0) == mhar.OK
    assert mhar.mhar_status_code(mhar.ST_STALL, 0) == mhar.OK
    assert mhar.mhar_status_code(mhar.ST_UNBOUNDED, 0) == mhar.E_UNBOUNDED
    assert mhar.mhar_status_code(mhar.ST_UNBOUNDED | mhar.ST_DRIFT, 0) == mhar.E_INFEASIBLE_DRIFT
    assert mhar.mhar_status_code(mhar.ST_DRIFT | mhar.ST_NONFINITE, 0) == mhar.E_NONFINITE
    assert mhar.mhar_status_code(mhar.ST_NONFINITE, 1) == mhar.E_TIMEOUT
    assert mhar.mhar_status_code(0, 1) == mhar.E_TIMEOUT
    assert mhar.mhar_strerror(mhar.E_TIMEOUT) == "MHAR_E_TIMEOUT"
    assert mhar.mhar_strerror(mhar.E_INFEASIBLE_DRIFT) == "MHAR_E_INFEASIBLE_DRIFT"


def test_built_for_sm103a_only():
    assert libbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
