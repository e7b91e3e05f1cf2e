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


def test_struct_layout_matches_header(lib):
    import ctypes
    # mhar_opts: u64 + 4 x i32 + pointer + i32 + 7 x i32 = 64 bytes on LP64.
    assert ctypes.sizeof(mhar.MharOpts) == 64
    assert ctypes.sizeof(mhar.MharStats) == 72


def test_built_for_sm103a_only():
    assert libbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
