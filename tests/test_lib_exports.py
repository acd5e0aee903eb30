"""The C-ABI library builds, loads without a GPU and exports every entry
point include/rca.h declares (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rca.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b((?:rca|ulm)_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2511_21647_gb300 import build
    return build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rca_create", "rca_set_stream", "rca_geometry_create", "rca_delay_tables",
                     "rca_beamform_projections", "ulm_localize", "rca_sync_status"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(\S+)", out))
    assert set(declared_functions()) <= exported


def test_binding_covers_every_declared_symbol(lib_path):
    from paper_2511_21647_gb300 import _lib, rca
    assert set(declared_functions()) == set(_lib.SIGNATURES)
    for n in declared_functions():
        assert callable(getattr(rca, n)), n


def test_host_side_status_strings_without_gpu(lib_path):
    from paper_2511_21647_gb300 import rca
    assert rca.rca_version() == (0 << 16) | 1
    assert rca.rca_status_string(0) == "ok"
    assert rca.rca_status_string(5) == "output capacity exceeded"


def test_struct_layouts_match_header():
    from paper_2511_21647_gb300 import _lib
    assert ctypes.sizeof(_lib.rca_geometry_desc) == 6 * 4 + 7 * 8 + 2 * 8
    assert ctypes.sizeof(_lib.ulm_params) == 40
    assert ctypes.sizeof(_lib.rca_bf_params) == 32
    assert _lib.LOC2D.itemsize == 40 and _lib.LOC3D.itemsize == 40
