"""The C-ABI library builds, loads and exports every symbol include/tdeig.h declares.

No compute calls: these run without a GPU.
"""
import ctypes
import os
import re
import subprocess

import pytest

from conftest import ROOT


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "tdeig.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(tdeig_\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def built():
    import __graft_entry__ as g
    g.build()
    from paper_1510_04591_gb300 import tdeig
    return tdeig


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("tdeig_create", "tdeig_solve", "tdeig_solve_batched", "tdeig_destroy",
              "tdeig_strerror", "tdeig_last_stats"):
        assert s in syms


def test_library_exports_every_declared_symbol(built):
    L = ctypes.CDLL(built.LIB_PATH)
    for s in declared_symbols():
        assert hasattr(L, s), s
    out = subprocess.run(["nm", "-D", "--defined-only", built.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (tdeig_\w+)", out))
    assert set(declared_symbols()) <= exported


def test_build_targets_sm103a_only():
    """The library is compiled for sm_103a alone (the device-side check of the
    loaded code, tdeig_binary_arch == 103, is a GPU test)."""
    from paper_1510_04591_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_strerror_and_defaults(built):
    assert built.strerror(0) == "success"
    assert "invalid" in built.strerror(-1)
    assert built.strerror(-99) == "unknown status"
    o = built.default_options()
    assert o.leaf == 32 and o.hss_threshold == 2000 and o.oversample == 10
    assert o.rank_cap == 100 and o.boundary_shift == 5 and o.tol == 1e-12


def test_null_arguments_rejected_without_gpu(built):
    L = built.lib()
    assert L.tdeig_create(None, None) == built.EINVAL
    assert L.tdeig_destroy(None) == built.EINVAL
    assert L.tdeig_solve(None, None, None, 4, None, None, 0) == built.EINVAL
    assert L.tdeig_last_stats(None, None, 0) == built.EINVAL


def test_oracle_is_not_imported_by_the_product():
    pkg = os.path.join(ROOT, "paper_1510_04591_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"(#|//).*", "", src).lower() or f == "inputs.py", f
