"""The C ABI: the library builds, loads, and exports every entry point that
include/kfac.h declares; host-side behaviour that needs no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libkfac():
    from paper_2206_15397_gb300 import build, kfac
    build.build()
    return kfac.lib()


def declared_entry_points():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"KFAC_API\s+[\w\s\*]+?\b(kfac_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for required in ("kfac_ea_update", "kfac_rsvd_invert", "kfac_precondition", "kfac_create", "kfac_destroy",
                     "kfac_get_status"):
        assert required in names


def test_every_declared_symbol_is_exported(libkfac):
    for name in declared_entry_points():
        assert hasattr(libkfac, name), name


def test_version_and_status_strings(libkfac):
    assert libkfac.kfac_version() >= 100
    assert libkfac.kfac_status_string(0) == b"KFAC_OK"
    assert libkfac.kfac_status_string(4) == b"KFAC_ERR_CHOLESKY"
    assert libkfac.kfac_status_string(999) == b"KFAC_ERR_UNKNOWN"


def test_null_arguments_rejected_without_device(libkfac):
    # Argument checks run on the host before any CUDA call.
    assert libkfac.kfac_create(None, 0, None) == 1
    assert libkfac.kfac_destroy(None) == 1
    assert libkfac.kfac_get_status(None, None) == 1
    assert libkfac.kfac_ea_update(None, 4, 4, None, 4, ctypes.c_float(0.9), 0, None, 4) == 1
    assert libkfac.kfac_ea_update_grouped(None, 1, None) == 1
    assert libkfac.kfac_precondition_grouped(None, 1, None) == 1
    assert libkfac.kfac_rsvd_invert_grouped(None, 1, None) == 1


def test_create_without_gpu_fails_loudly(libkfac):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = libkfac.kfac_create(ctypes.byref(h), 0, None)
    assert st != 0 and not h.value
