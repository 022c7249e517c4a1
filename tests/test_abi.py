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


def _c_layout(structs):
    """sizeof and offsetof of each struct field as the C compiler lays out include/ie.h (gcc, host)."""
    import shutil
    import subprocess
    import tempfile

    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ie.h"', "int main(void) {"]
    for st, fields in structs.items():
        lines.append(f'  printf("{st} size %zu\\n", sizeof({st}));')
        for f in fields:
            lines.append(f'  printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines))
        subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    res = {}
    for line in out.splitlines():
        st, key, val = line.split()
        res[(st, key)] = int(val)
    return res


def test_binding_structs_match_the_header_layout():
    """The ctypes mirrors of ie_grid, ie_dipole, ie_opts, ie_info and ie_batch_item have the sizes and field
    offsets the C compiler gives the header's structs (a field added on one side only fails here)."""
    from paper_2306_17537_gb300 import build

    if not os.path.exists(build.LIB):
        pytest.skip("library not built")
    from paper_2306_17537_gb300 import ie

    mirrors = {"ie_grid": ie.ie_grid, "ie_dipole": ie.ie_dipole, "ie_opts": ie.ie_opts, "ie_info": ie.ie_info,
               "ie_batch_item": ie.ie_batch_item}
    structs = {name: [f[0] for f in cls._fields_] for name, cls in mirrors.items()}
    c = _c_layout(structs)
    for name, cls in mirrors.items():
        assert ctypes.sizeof(cls) == c[(name, "size")], name
        for fname in structs[name]:
            assert getattr(cls, fname).offset == c[(name, fname)], (name, fname)
