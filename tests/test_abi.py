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
    assert libpmc.pmc_surrogate_infer(None, None, 1, None) == -1
    assert libpmc.pmc_debug_surrogate_waits(None) == -1
    libpmc.pmc_debug_drain_waits.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64]
    assert libpmc.pmc_debug_drain_waits(None, 10, 1) == -1
    assert libpmc.pmc_enable_profile(None, 2) == -1
    libpmc.pmc_enable_deposit_log.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
    assert libpmc.pmc_enable_deposit_log(None, 10) == -1
    assert libpmc.pmc_read_deposit_log(None, None, 0, None) == -1


def test_create_rejects_bad_options_before_touching_a_device(libpmc):
    """Option checks that need no GPU: the statistical group count, and allocator hooks that
    come without their partner (a block from a caller's allocator must not reach cudaFree)."""
    from paper_1409_8336_gb300 import engine

    libpmc.pmc_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    ctx = ctypes.c_void_p()
    keep = engine.AllocFn(lambda n, user: None)
    for n_batches, alloc in ((1, None), (1025, None), (10, keep)):
        o = engine.Options()
        o.n_batches = n_batches
        if alloc is not None:
            o.alloc = alloc
        assert libpmc.pmc_create(ctypes.byref(ctx), ctypes.byref(o)) == -1
        assert not ctx.value


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


def test_gamma_plan_counts_the_search_sphere(libpmc):
    """Host logic of the gamma entry points (no device call): a plan holds a 256-byte head
    and 16 bytes per voxel offset within the search sphere; bad arguments are refused."""
    d = ctypes.c_double
    libpmc.pmc_gamma_plan_bytes.argtypes = [d, d, d, d, d, ctypes.POINTER(ctypes.c_size_t)]
    nb = ctypes.c_size_t(0)
    for voxel, dta, search in (((0.1, 0.1, 0.1), 2.0, 0.0), ((0.125, 0.125, 0.25), 2.0, 0.0),
                               ((0.05, 0.1, 0.2), 3.0, 5.0)):
        assert libpmc.pmc_gamma_plan_bytes(*voxel, dta, search, ctypes.byref(nb)) == 0
        r = search if search > 0 else 1.5 * dta
        h = [v * 10.0 for v in voxel]
        m = [int(r // x) + 1 for x in h]
        count = sum(1 for i in range(-m[0], m[0] + 1) for j in range(-m[1], m[1] + 1) for k in range(-m[2], m[2] + 1)
                    if (i * h[0]) ** 2 + (j * h[1]) ** 2 + (k * h[2]) ** 2 <= r * r)
        assert nb.value == 256 + 16 * count
    assert libpmc.pmc_gamma_plan_bytes(0.1, 0.1, 0.1, 2.0, 0.0, None) == -1
    assert libpmc.pmc_gamma_plan_bytes(0.1, -0.1, 0.1, 2.0, 0.0, ctypes.byref(nb)) == -1
    assert libpmc.pmc_gamma_plan_bytes(0.1, 0.1, 0.1, 0.0, 0.0, ctypes.byref(nb)) == -1
    assert libpmc.pmc_gamma_plan_bytes(0.001, 0.001, 0.001, 2.0, 30.0, ctypes.byref(nb)) == -1   # sphere too large
    vp, i = ctypes.c_void_p, ctypes.c_int
    libpmc.pmc_gamma_plan.argtypes = [d, d, d, d, d, vp, ctypes.c_size_t, vp]
    libpmc.pmc_gamma_device.argtypes = [vp, vp, vp, i, i, i, d, d, vp, vp]
    # refused before any device call: no plan memory, a misaligned or short plan, NULL doses,
    # an empty grid, a non-positive dose criterion
    assert libpmc.pmc_gamma_plan(0.1, 0.1, 0.1, 2.0, 0.0, None, 4096, None) == -1
    assert libpmc.pmc_gamma_plan(0.1, 0.1, 0.1, 2.0, 0.0, 260, 4096, None) == -1
    assert libpmc.pmc_gamma_plan(0.1, 0.1, 0.1, 2.0, 0.0, 256, 512, None) == -1
    assert libpmc.pmc_gamma_device(256, None, None, 4, 4, 4, 2.0, 0.1, None, None) == -1
    assert libpmc.pmc_gamma_device(256, 512, 1024, 0, 4, 4, 2.0, 0.1, None, None) == -1
    assert libpmc.pmc_gamma_device(260, 512, 1024, 4, 4, 4, 2.0, 0.1, None, None) == -1
    assert libpmc.pmc_gamma_device(256, 512, 1024, 4, 4, 4, 0.0, 0.1, None, None) == -1


def test_binding_loads_and_declares_every_entry_point():
    """The Python binding loads both builds and sets the argument types of every export
    (no device call)."""
    from paper_1409_8336_gb300 import build, engine

    build.build()
    for path in (engine.LIB_PATH, engine.LIB_FAST_PATH):
        L = engine.lib(path)
        for name in engine.EXPORTS:
            assert getattr(L, name).argtypes is not None or name in ("pmc_last_error",), name
