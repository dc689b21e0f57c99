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
    assert libkfac.kfac_draw_omega(None, 4, 4, ctypes.c_uint64(1), None, 4) == 1


def test_create_without_gpu_fails_loudly(libkfac):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = libkfac.kfac_create(ctypes.byref(h), 0, None)
    assert st != 0 and not h.value


def _param_class(decl: str) -> str:
    decl = " ".join(decl.split())
    if "*" in decl:
        return "ptr"
    if "unsigned long long" in decl or "uint64_t" in decl:
        return "u64"
    if "long long" in decl or "int64_t" in decl or "size_t" in decl:
        return "i64"
    if decl.startswith("float") or decl.startswith("const float"):
        return "f32"
    if decl.startswith("double") or decl.startswith("const double"):
        return "f64"
    return "i32"


def _ctype_class(t) -> str:
    if t in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(t, "_type_") and isinstance(t._type_, type):
        return "ptr"
    if t is ctypes.c_float:
        return "f32"
    if t is ctypes.c_double:
        return "f64"
    size = ctypes.sizeof(t)
    unsigned = t(-1).value > 0
    return {(8, True): "u64", (8, False): "i64", (4, False): "i32"}.get((size, unsigned), "?")


def test_binding_argtypes_match_the_header(libkfac):
    """Every argtypes list the binding declares has the header prototype's
    parameter count and kinds (a mismatch would pass wrong values silently)."""
    text = open(os.path.join(ROOT, "include", "kfac.h")).read()
    protos = dict(re.findall(r"KFAC_API\s+[\w\s\*]+?\b(kfac_\w+)\s*\(([^)]*)\)", text))
    checked = 0
    for name, params in protos.items():
        fn = getattr(libkfac, name)
        if fn.argtypes is None:
            continue
        decls = [p.strip() for p in params.split(",") if p.strip() and p.strip() != "void"]
        want = [_param_class(p) for p in decls]
        got = [_ctype_class(t) for t in fn.argtypes]
        assert got == want, (name, got, want)
        checked += 1
    assert checked >= 20, checked
