"""The C-ABI library loads and exports every entry point that include/ie.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("ie.h", "ie_fno.h")]


def declared_symbols():
    text = "".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ie_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2306_17537_gb300 import build

    if not os.path.exists(build.LIB):
        try:
            build.build()
        except RuntimeError as e:  # no nvcc on this machine
            pytest.skip(f"cannot build the library here: {e}")
    return build.LIB


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("ie_create", "ie_set_contrast", "ie_solve", "ie_destroy", "ie_last_error", "ie_matvec",
                 "ie_gmres", "ie_green_spectrum", "ie_incident_field", "ie_receiver_fields"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib_path):
    from paper_2306_17537_gb300 import ie

    assert sorted(ie.EXPORTED) == declared_symbols()


def test_create_rejects_bad_arguments_without_touching_the_gpu(lib_path):
    from paper_2306_17537_gb300 import ie

    for args in [(0, 4, 4, 0.5, 0.1, 1e5), (4, 4, 4, -0.5, 0.1, 1e5), (4, 4, 4, 0.5, 0.0, 1e5),
                 (4, 4, 4, 0.5, 0.1, float("nan")), (4, 4, 600, 0.5, 0.1, 1e5)]:
        nx, ny, nz, h, s0, f = args
        g = ie.ie_grid(nx, ny, nz, (ctypes.c_double * 3)(0, 0, 0))
        p = ctypes.c_void_p()
        st = ie._lib.ie_create(ctypes.byref(g), h, s0, f, ctypes.byref(p))
        assert st == ie.IE_EINVAL and not p.value
    assert ie._lib.ie_last_error(None) == b"null context"
