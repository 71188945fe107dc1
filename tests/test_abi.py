"""The C-ABI library builds, loads and exports every entry point include/pmc.h declares (CPU only:
no compute call is made)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(pmc_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpmc():
    from paper_1409_8336_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pmc_create", "pmc_destroy", "pmc_load_materials", "pmc_load_phantom", "pmc_add_spots",
                     "pmc_transport", "pmc_read_dose", "pmc_read_ledger", "pmc_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libpmc):
    missing = [n for n in declared_functions() if not hasattr(libpmc, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_1409_8336_gb300 import engine

    assert set(declared_functions()) <= set(engine.EXPORTS)


def test_invalid_calls_fail_without_a_device(libpmc):
    libpmc.pmc_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert libpmc.pmc_create(None, None) == -1          # PMC_E_INVALID, no context pointer
    libpmc.pmc_transport.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p]
    assert libpmc.pmc_transport(None, 10, 1, 0, None) == -1


def test_oracle_and_engine_share_no_code():
    """The CUDA path and the oracle are independent: neither includes nor imports the other."""
    csrc = os.path.join(ROOT, "paper_1409_8336_gb300", "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f)).read()
        assert "oracle" not in text.lower()
    for f in ("engine.py", "build.py", "__init__.py", "workloads.py"):
        text = open(os.path.join(ROOT, "paper_1409_8336_gb300", f)).read()
        assert "import oracle" not in text and "from oracle" not in text
    for f in ("oracle.c", "oracle.py"):
        text = open(os.path.join(ROOT, "oracle", f)).read()
        assert "paper_1409_8336_gb300" not in text and "pmc_device" not in text
