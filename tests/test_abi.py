"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/mfa.h declares (no compute call is made here)."""
import os
import re
import subprocess

import pytest

from paper_2210_06528_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "mfa.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mfa_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib_path():
    return B.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["mfa_encode", "mfa_schwarz_iterate", "mfa_decode", "mfa_residual", "mfa_create",
                     "mfa_destroy", "mfa_get_ctrl", "mfa_free", "mfa_sync", "mfa_interface_jumps"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_and_status_strings(lib_path):
    from paper_2210_06528_gb300 import mfa
    lib = mfa.load(lib_path)
    for n in declared_functions():
        assert hasattr(lib, n)
    assert mfa.status_string(mfa.MFA_OK) == "ok"
    assert "layout" in mfa.status_string(mfa.MFA_ERR_LAYOUT)
    assert mfa.status_string(12345) == "unknown status"


def test_binding_exports_c_names():
    from paper_2210_06528_gb300 import mfa
    for n in declared_functions():
        if n == "mfa_status_string":
            continue
        assert callable(getattr(mfa, n)), n


def test_layout_struct_matches_header_size(lib_path):
    """ctypes mirrors of mfa_layout / mfa_report have the C sizes."""
    import ctypes
    from paper_2210_06528_gb300 import mfa
    # dim, degree (8) + npts (24) + nspans, nsub (24) + 3 pointers (24) + overlap (12) + precision (4) + lo, hi
    # (48) + knots (4, then 4 of padding) + 3 weight pointers (24)
    assert ctypes.sizeof(mfa.mfa_layout) == 8 + 24 + 24 + 24 + 12 + 4 + 48 + 8 + 24
    # iters, status (8) + 5 doubles + jump_orders and padding (8) + jump_deriv (8 doubles)
    assert ctypes.sizeof(mfa.mfa_report) == 8 + 5 * 8 + 8 + 8 * 8


def test_no_oracle_import_in_product():
    """The product package never imports or loads the oracle."""
    pkg = os.path.join(ROOT, "paper_2210_06528_gb300")
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b)|oracle[/.]mfa_oracle", re.M)
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not pat.search(src), f
